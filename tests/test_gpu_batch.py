"""Batched path (persistent raster / backward over an item table, CUDA graph) against the per-item path and
against the FP64 oracle."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2405_02508_gb300 import scenes

from . import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def orc():
    import oracle

    oracle.build()
    return oracle


def _multiview_batch(n_views=6, H=512, W=384, n=48, tile=32):
    import torch

    from paper_2405_02508_gb300.batch import BatchRenderer

    sc = scenes.head_multiview(n_views=n_views, H=H, W=W, n=n, tex_size=256)
    meshes = [(sc.verts, sc.tris)]
    items = [(0, v, H, W) for v in range(n_views)]
    tex = torch.from_numpy(sc.tex).cuda()
    br = BatchRenderer(meshes, items, sc.cams, sc.shading, 2, tex, tile=tile)
    return sc, br, tex


@pytest.mark.parametrize("tile", [16, 32, 64])
def test_batch_equals_multiview_renderer(tile):
    """Views of one mesh as batch items give the same index and image as the multi-view entry points and the
    same gradients up to summation order."""
    import torch

    sc, br, tex = _multiview_batch(tile=tile)
    verts = torch.from_numpy(sc.verts).cuda()
    attr = torch.from_numpy(sc.attr).cuda()
    g = torch.from_numpy(sc.upstream()).cuda()
    br.prepare(verts, attr, tex)
    br.backward(g.reshape(-1, sc.shading.C), attr, tex)
    br.check()
    ref = parity.gpu_run(sc, sc.upstream(), tile=tile if tile != 64 else 32)
    n, H, W = sc.n_views, sc.H, sc.W
    np.testing.assert_array_equal(br.index.cpu().numpy().reshape(n, H, W), ref.index)
    np.testing.assert_array_equal(br.image.cpu().numpy().reshape(n, H, W, -1), ref.image)
    gv = br.grad_vpix.cpu().numpy().reshape(n, -1, 3)
    np.testing.assert_allclose(gv, ref.grad_vpix, rtol=1e-5, atol=1e-6 * np.abs(ref.grad_vpix).max())
    np.testing.assert_allclose(br.grad_verts.cpu().numpy(), ref.grad_verts, rtol=1e-4,
                               atol=1e-6 * np.abs(ref.grad_verts).max())


@pytest.mark.parametrize("tile", [16, 64])
def test_fused_render_equals_raster_then_shade(tile):
    """mer_batch_render (raster + shade in one pass) writes the same index, depth, barycentrics and image as
    mer_batch_rasterize followed by mer_batch_shade, bit for bit, and the same cover image; also with
    interpolated attributes."""
    import torch

    from paper_2405_02508_gb300.batch import BatchRenderer

    sc, br, tex = _multiview_batch(n_views=3, H=300, W=260, n=40, tile=tile)
    verts = torch.from_numpy(sc.verts).cuda()
    attr = torch.from_numpy(sc.attr).cuda()
    br.prepare(verts, attr, tex)  # sizes the bin lists
    P = br.index.numel()
    out = {}
    for fused in (False, True):
        depth = torch.full((P,), -7.0, device="cuda")
        bary = torch.full((P, 2), -7.0, device="cuda")
        br.index.fill_(-9)
        br.image.fill_(-9.0)
        br.cover.fill_(255)
        br.forward(verts, attr, tex, depth, bary, fused=fused)
        br.check()
        out[fused] = (br.index.clone(), br.image.clone(), depth, bary, br.cover.clone())
    for a, b in zip(out[False], out[True]):  # the cover image too
        assert torch.equal(a, b)
    its = scenes.uneven_batch(n_items=5, t_max=20000, resolutions=(96, 200))
    br2 = BatchRenderer([(it.verts, it.tris) for it in its], [(k, k, it.H, it.W) for k, it in enumerate(its)],
                        np.concatenate([it.cams for it in its]), its[0].shading, 3, None, tile=tile)
    v2 = torch.from_numpy(np.concatenate([it.verts for it in its])).cuda()
    a2 = torch.from_numpy(np.concatenate([it.attr for it in its])).cuda()
    br2.prepare(v2, a2)
    imgs = []
    for fused in (False, True):
        br2.image.fill_(-9.0)
        br2.forward(v2, a2, fused=fused)
        br2.check()
        imgs.append((br2.index.clone(), br2.image.clone()))
    assert torch.equal(imgs[0][0], imgs[1][0]) and torch.equal(imgs[0][1], imgs[1][1])


def test_batch_uneven_items_against_oracle(orc):
    """Items of the uneven batch (different meshes, triangle counts and resolutions) in one batched pass;
    every sampled item matches the oracle at the parity tolerances."""
    import torch

    from paper_2405_02508_gb300.batch import BatchRenderer

    its = scenes.uneven_batch(n_items=24, t_max=40000)
    meshes = [(it.verts, it.tris) for it in its]
    cams = np.concatenate([it.cams for it in its])
    items = [(k, k, it.H, it.W) for k, it in enumerate(its)]
    sh = its[0].shading
    br = BatchRenderer(meshes, items, cams, sh, 3, None, tile=32)
    verts = torch.from_numpy(np.concatenate([it.verts for it in its])).cuda()
    attr = torch.from_numpy(np.concatenate([it.attr for it in its])).cuda()
    grads = [it.upstream()[0] for it in its]
    g = torch.from_numpy(np.concatenate([x.reshape(-1, sh.C) for x in grads])).cuda()
    br.prepare(verts, attr)
    br.backward(g, attr)
    br.check()
    for k in (0, 5, 11, 23):
        it = its[k]
        ov = orc.render(it)[0]
        gs, _, cnt, S = orc.backward(ov.scr, ov.snap, ov.flags, it.tris, ov.index, ov.image, grads[k], it.attr, sh,
                                     want_abs=True)
        gi = br.item_index(k).cpu().numpy()
        assert np.all((gi == ov.index) | ov.tie)
        np.testing.assert_allclose(br.item_image(k).cpu().numpy(), ov.image, rtol=parity.IMG_TOL, atol=parity.IMG_TOL)
        ex = parity.excluded_vertices(it.tris, gi, ov.index)
        nbad, worst = parity.grad_violations(br.item_grad_vpix(k).cpu().numpy(), gs, S, ex)
        assert nbad == 0, (k, worst)


def test_full_uneven_batch_in_bench_configuration(orc):
    """The whole 256-mesh uneven batch (500..200k triangles, 128^2..1024^2) in one batched pass with the
    bench's 32 px tile and default grid; the smallest, the largest and two middle items against the oracle."""
    import torch

    from paper_2405_02508_gb300.batch import BatchRenderer

    its = scenes.uneven_batch(n_items=256)
    sh = its[0].shading
    br = BatchRenderer([(it.verts, it.tris) for it in its], [(k, k, it.H, it.W) for k, it in enumerate(its)],
                       np.concatenate([it.cams for it in its]), sh, 3, None, tile=32)
    verts = torch.from_numpy(np.concatenate([it.verts for it in its])).cuda()
    attr = torch.from_numpy(np.concatenate([it.attr for it in its])).cuda()
    grads = {}
    br.prepare(verts, attr)
    T = np.array([len(it.tris) for it in its])
    order = np.argsort(T)
    picks = [int(order[0]), int(order[85]), int(order[170]), int(order[-1])]
    g = torch.zeros((int(br.tot.pixels), sh.C), device="cuda")
    for k in picks:
        p0, H, W = br.item_pix[k]
        grads[k] = its[k].upstream()[0]
        g[p0:p0 + H * W] = torch.from_numpy(grads[k].reshape(-1, sh.C)).cuda()
    br.backward(g, attr)
    br.check()
    for k in picks:
        it = its[k]
        ov = orc.render(it)[0]
        gs, _, cnt, S = orc.backward(ov.scr, ov.snap, ov.flags, it.tris, ov.index, ov.image, grads[k], it.attr, sh,
                                     want_abs=True)
        gi = br.item_index(k).cpu().numpy()
        assert np.all((gi == ov.index) | ov.tie)
        np.testing.assert_allclose(br.item_image(k).cpu().numpy(), ov.image, rtol=parity.IMG_TOL, atol=parity.IMG_TOL)
        ex = parity.excluded_vertices(it.tris, gi, ov.index)
        nbad, worst = parity.grad_violations(br.item_grad_vpix(k).cpu().numpy(), gs, S, ex)
        assert nbad == 0, (k, worst)


def test_batch_graph_replay_matches_eager():
    import torch

    sc, br, tex = _multiview_batch(n_views=4, H=256, W=320, n=32)
    verts = torch.from_numpy(sc.verts).cuda()
    attr = torch.from_numpy(sc.attr).cuda()
    g = torch.from_numpy(sc.upstream()).cuda().reshape(-1, sc.shading.C)
    br.prepare(verts, attr, tex)
    br.step(verts, attr, g, tex)
    br.check()
    idx0 = br.index.clone()
    gw0 = br.grad_verts.clone()
    br.capture(verts, attr, g, tex)
    for _ in range(3):
        br.index.fill_(-5)
        br.replay()
    torch.cuda.synchronize()
    br.check()
    assert torch.equal(br.index, idx0)
    np.testing.assert_allclose(br.grad_verts.cpu().numpy(), gw0.cpu().numpy(), rtol=1e-4,
                               atol=1e-6 * float(gw0.abs().max()))


def test_autotune_picks_a_candidate():
    import torch

    from paper_2405_02508_gb300.batch import BatchRenderer, autotune_tile

    sc = scenes.head_multiview(n_views=2, H=256, W=256, n=24, tex_size=64)
    tex = torch.from_numpy(sc.tex).cuda()
    verts = torch.from_numpy(sc.verts).cuda()
    attr = torch.from_numpy(sc.attr).cuda()
    g = torch.from_numpy(sc.upstream()).cuda().reshape(-1, sc.shading.C)

    def make(tile):
        br = BatchRenderer([(sc.verts, sc.tris)], [(0, 0, 256, 256), (0, 1, 256, 256)], sc.cams, sc.shading, 2, tex,
                           tile=tile)
        br.prepare(verts, attr, tex)
        return br

    best, times = autotune_tile(make, lambda r: r.step(verts, attr, g, tex), cache_file=None)
    assert best in (16, 32, 64) and set(times) == {16, 32, 64}
    from paper_2405_02508_gb300.batch import autotune

    def make2(tile, ctas):
        br = make(tile)
        br.persistent_ctas = ctas
        return br

    tile, ctas, t2 = autotune(make2, lambda r: r.step(verts, attr, g, tex), tiles=(16, 32), cache_file=None)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert tile in (16, 32) and ctas in (sms, 2 * sms, 4 * sms) and len(t2) == 6
