"""The deterministic option (MER_DETERMINISTIC with FP64 shading) against the oracle at the stated bound, and
its reproducibility.

With the option, every per-pixel quantity is FP64 and the sums are exact fixed-point sums, so the vertex
gradients must meet |g - o| <= 1e-6 + 1e-4 |o| per component on every configuration with no conditioning
term, and the image must be the oracle's image correctly rounded to FP32.  The results must also be bitwise
identical from run to run, with the barycentric image stored or recomputed, at every bin tile, and between
the per-view and the batched entry points (vertex-record gradients).
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_2405_02508_gb300 import scenes
from paper_2405_02508_gb300.scenes import Scene

from . import parity
from .test_gpu_parity import CASES, run_parity

pytestmark = pytest.mark.gpu

ALL = 7
DET = 16


@pytest.fixture(scope="module")
def orc():
    import oracle

    oracle.build()
    return oracle


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2405_02508_gb300 import binding

    binding.lib()


# ---------------------------------------------------------------------------
# the five workloads at the stated bound
# ---------------------------------------------------------------------------

def test_det_tiny_icosphere_l2(orc):
    sc = scenes.tiny_icosphere()
    tgt = Scene(sc.name, sc.target_verts, sc.tris, sc.cams, sc.H, sc.W, sc.attr, sc.shading)
    It = orc.render(tgt)[0].image
    Io = orc.render(sc)[0].image
    g = (2.0 * (Io - It))[None].astype(np.float32)
    run_parity(orc, sc, g, terms=ALL | DET, want_attr=True, label="c1 tiny L2")


@pytest.mark.parametrize("tile", [8, 32])
def test_det_intersection_two_spheres(orc, tile):
    sc = scenes.two_spheres()
    _, _, counts = run_parity(orc, sc, sc.upstream(), terms=ALL | DET, tile=tile, label=f"c2 two spheres t{tile}")
    assert counts[0]["intersection"] > 50


def test_det_intersections_off_and_single_terms(orc):
    sc = scenes.two_spheres(H=256, W=256)
    run_parity(orc, sc, sc.upstream(), terms=1 | 2 | DET, label="c2 intersections off")
    run_parity(orc, sc, sc.upstream(), terms=1 | 4 | DET, label="c2 edge only")
    run_parity(orc, sc, sc.upstream(), terms=2 | DET, label="c2 interior only")


@pytest.mark.parametrize("scene", ["tiny", "two_spheres", "open_sphere"])
def test_det_exact_crossing_option(orc, scene):
    sc = {"tiny": lambda: scenes.tiny_icosphere(),
          "two_spheres": lambda: scenes.two_spheres(H=256, W=256, subdiv=4),
          "open_sphere": lambda: scenes.open_sphere(H=256, W=256)}[scene]()
    run_parity(orc, sc, sc.upstream(), terms=ALL | 8 | DET, label=f"exact crossing {scene}")


def test_det_backface_image(orc):
    sc = scenes.open_sphere(H=256, W=256)
    run_parity(orc, sc, sc.upstream(), terms=ALL | DET, want_attr=True, label="back-face image")


@pytest.mark.parametrize("store_bary", [True, False])
def test_det_head_single_view(orc, store_bary):
    sc = scenes.head_single_view()
    run_parity(orc, sc, sc.upstream(), terms=ALL | DET, want_attr=True, store_bary=store_bary,
               label=f"c3 head 1024 bary={'stored' if store_bary else 'recomputed'}")


def test_det_multiview_full_size_sampled_views(orc):
    sc = scenes.head_multiview()
    run_parity(orc, sc, sc.upstream(), terms=ALL | DET, views=[0, 13, 31], check_world=False,
               label="c4 32x1334x2048 sampled")


def test_det_uneven_items(orc):
    items = scenes.uneven_batch(n_items=256)
    T = np.array([len(it.tris) for it in items])
    order = np.argsort(T)
    stats = []
    for i in [order[0], order[len(order) // 3], order[2 * len(order) // 3], order[-1]]:
        it = items[i]
        stats += run_parity(orc, it, it.upstream(), terms=ALL | DET, label=f"c5 item {i}", tie_check=False)[1]
    parity.assert_tie_share(stats)


@pytest.mark.parametrize("case", sorted(CASES))
def test_det_edge_cases(orc, case):
    """The edge-case scenes (ragged, 1x1, strips, full screen, background only, guard band, behind the camera,
    degenerate triangles, centres on edges) at the stated bound."""
    import torch

    from paper_2405_02508_gb300 import binding as B
    from paper_2405_02508_gb300.render import Renderer

    scr, tris, H, W, sh, attr = CASES[case]
    g = np.random.default_rng(1).standard_normal((1, H, W, 1)).astype(np.float32)
    r = Renderer(torch.from_numpy(tris), len(scr), 1, H, W, sh, attr.shape[1], tile=16, precise=True)
    r.project_screen(torch.from_numpy(scr[None]).cuda())
    r.rasterize()
    a = torch.from_numpy(attr).cuda()
    r.shade(a, None)
    r.grad_vpix.zero_()
    r._ensure_backward_workspace(ALL | DET, None)
    B.mer_backward(r.vpix, r.tris, r.index, r.image, torch.from_numpy(g).cuda(), a, None, r.sh, ALL | DET,
                   r.grad_vpix, None, r.workspace)
    r.check_status()
    gi, gg = r.index[0].cpu().numpy(), r.grad_vpix[0].cpu().numpy()
    s, snap, flags = orc.snap_screen(scr)
    oi, tie, _ = orc.rasterize(s, snap, flags, tris, H, W)
    img = orc.shade(s, tris, oi, attr, sh)
    og, _, _, _ = orc.backward(s, snap, flags, tris, oi, img.astype(np.float32).astype(np.float64), g[0], attr, sh,
                               mode=ALL, want_abs=True)
    assert np.all((gi == oi) | tie)
    _, far = parity.image_rounding_mismatches(r.image[0].cpu().numpy()[gi == oi], img[gi == oi])
    assert not far.any()  # FP64 shading rounded once: within one FP32 ulp of the oracle's FP64 value
    nbad, worst = parity.grad_violations(gg, og, None, parity.excluded_vertices(tris, gi, oi), 0.0)
    assert nbad == 0, worst


# ---------------------------------------------------------------------------
# reproducibility
# ---------------------------------------------------------------------------

def test_det_bitwise_recompute_runs_and_tiles():
    """Through the autograd function: stored or recomputed barycentrics, repeated runs and bin tiles 8/16/32 give
    the same vertex and attribute gradient bits."""
    import torch

    from paper_2405_02508_gb300 import binding as B
    from paper_2405_02508_gb300.render import MerRender, Renderer

    sc = scenes.head_single_view(H=384, W=320, n=48, tex_size=256)
    tex = torch.from_numpy(sc.tex).cuda()
    cams = B.cameras_tensor(sc.cams)
    g = torch.from_numpy(sc.upstream()).cuda()
    out = []
    for tile, recompute in [(16, True), (16, False), (16, True), (8, False), (32, True)]:
        r = Renderer(torch.from_numpy(sc.tris), len(sc.verts), 1, sc.H, sc.W, sc.shading, 2, tex.shape, tile=tile,
                     precise=True)
        r.terms = ALL | DET
        verts = torch.from_numpy(sc.verts).cuda().requires_grad_(True)
        attr = torch.from_numpy(sc.attr).cuda().requires_grad_(True)
        img = MerRender.apply(verts, attr, tex, cams, r, recompute)
        (img * g).sum().backward()
        r.check_status()
        out.append((img.detach().cpu().numpy(), verts.grad.cpu().numpy(), attr.grad.cpu().numpy()))
    for k in range(1, len(out)):
        for a, b in zip(out[0], out[k]):
            assert a.tobytes() == b.tobytes()
    assert np.abs(out[0][1]).max() > 0


def test_det_batched_equals_per_view_bitwise():
    """The batched entry points with MER_DETERMINISTIC give the per-view entry points' vertex-record gradient
    bits, at every bin tile and persistent grid, and the same world gradients from run to run."""
    import torch

    from paper_2405_02508_gb300 import binding as B
    from paper_2405_02508_gb300.batch import BatchRenderer

    sc = scenes.head_multiview(n_views=5, H=300, W=240, n=40, tex_size=128)
    n, H, W, C = sc.n_views, sc.H, sc.W, sc.shading.C
    ref = parity.gpu_run(sc, sc.upstream(), terms=ALL | DET)
    verts = torch.from_numpy(sc.verts).cuda()
    attr = torch.from_numpy(sc.attr).cuda()
    tex = torch.from_numpy(sc.tex).cuda()
    g = torch.from_numpy(sc.upstream()).cuda().reshape(-1, C)
    worlds = []
    for tile, ctas in [(16, 0), (64, 152), (32, 600)]:
        br = BatchRenderer([(sc.verts, sc.tris)], [(0, v, H, W) for v in range(n)], sc.cams, sc.shading,
                           sc.attr.shape[1], tex, tile=tile, persistent_ctas=ctas, precise=True)
        br.prepare(verts, attr, tex)
        br.backward(g, attr, tex, terms=ALL | DET)
        br.check()
        gv = br.grad_vpix.cpu().numpy().reshape(n, -1, 3)
        assert gv.tobytes() == ref.grad_vpix.tobytes()
        assert br.image.cpu().numpy().reshape(n, H, W, C).tobytes() == ref.image.tobytes()
        worlds.append(br.grad_verts.cpu().numpy())
    for w in worlds[1:]:
        assert w.tobytes() == worlds[0].tobytes()
    np.testing.assert_allclose(worlds[0], ref.grad_verts, rtol=1e-6, atol=1e-7)


def test_det_fixed_point_range_reported():
    """A contribution beyond the fixed-point range (an upstream gradient of 1e12) sets MER_EFIXED; the status
    clears and a normal call runs clean afterwards."""
    import torch

    from paper_2405_02508_gb300 import binding as B
    from paper_2405_02508_gb300.render import Renderer

    sc = scenes.tiny_icosphere()
    r = Renderer(torch.from_numpy(sc.tris), len(sc.verts), 1, sc.H, sc.W, sc.shading, 3, precise=True)
    cams = B.cameras_tensor(sc.cams)
    attr = torch.from_numpy(sc.attr).cuda()
    r.forward(torch.from_numpy(sc.verts).cuda(), cams, attr)
    huge = torch.full((1, sc.H, sc.W, sc.shading.C), 1e12, device="cuda")
    r.backward(huge, cams, attr, terms=ALL | DET)
    with pytest.raises(B.MerError) as e:
        r.check_status()
    assert e.value.code == B.MER_EFIXED
    r.backward(torch.from_numpy(sc.upstream()).cuda(), cams, attr, terms=ALL | DET)
    r.check_status()


def test_det_requires_workspace():
    import torch

    from paper_2405_02508_gb300 import binding as B
    from paper_2405_02508_gb300.render import Renderer

    sc = scenes.tiny_icosphere()
    r = Renderer(torch.from_numpy(sc.tris), len(sc.verts), 1, sc.H, sc.W, sc.shading, 3, precise=True)
    attr = torch.from_numpy(sc.attr).cuda()
    r.forward(torch.from_numpy(sc.verts).cuda(), B.cameras_tensor(sc.cams), attr)
    g = torch.from_numpy(sc.upstream()).cuda()
    small = torch.zeros(64, device="cuda")  # 256 bytes: the status header only
    with pytest.raises(B.MerError) as e:
        B.mer_backward(r.vpix, r.tris, r.index, r.image, g, attr, None, r.sh, ALL | DET, r.grad_vpix, None, small)
    assert e.value.code == B.MER_EINVAL
    with pytest.raises(B.MerError):
        B.mer_backward(r.vpix, r.tris, r.index, r.image, g, attr, None, r.sh, ALL | DET, r.grad_vpix, None, None)
