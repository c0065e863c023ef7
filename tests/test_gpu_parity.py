"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle, element by element.

The tolerances are stated in ``tests/parity.py``.  Scenes are the five workloads
(tiny icosphere, interpenetrating spheres, head-scale single view, 32-view
multi-view at full size with sampled oracle views, uneven batch items) plus
edge cases: empty meshes, ragged and degenerate image sizes, all-background
views, triangles behind the camera or far outside the image, and every bin
tile size.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_2405_02508_gb300 import scenes
from paper_2405_02508_gb300.scenes import Scene, Shading

from . import parity

pytestmark = pytest.mark.gpu

ALL = 7


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


DET = 16  # MER_DETERMINISTIC


def run_parity(orc, scene, grads, views=None, terms=ALL, tile=16, check_world=True, want_attr=False,
               store_bary=True, cover_hint=True, label=None, tie_check=True):
    """The scene through the CUDA path and the oracle, every compared view element by element (and the world
    and attribute gradients when every view is compared).  With DET in ``terms``: FP64 shading and the
    deterministic backward on the GPU, the oracle's image rounded to FP32 as its edge-step input, and the
    stated gradient bound with no conditioning term."""
    det = bool(terms & DET)
    gpu = parity.gpu_run(scene, grads, terms=terms, tile=tile, want_attr=want_attr, store_bary=store_bary,
                         cover_hint=cover_hint)
    views = list(range(scene.n_views)) if views is None else list(views)
    ovs = orc.render(scene, views)
    gs, gw, counts, ga = orc.backward_scene(scene, ovs, [grads[v] for v in views], views, mode=terms & 15,
                                            want_attr=want_attr,
                                            images=[parity.oracle_image(ov, det) for ov in ovs])
    label = label or scene.name
    stats = []
    for k, v in enumerate(views):
        stats.append(parity.compare_view(gpu, v, ovs[k], gs[k], scene.tris, S=counts[k]["grad_abs"],
                                         deterministic=det, label=label))
    if tie_check:
        parity.assert_tie_share(stats)
    ex = np.unique(np.concatenate([parity.excluded_vertices(scene.tris, gpu.index[v], ovs[k].index,
                                                            parity.ambiguous(ovs[k], det))
                                   for k, v in enumerate(views)]))
    cond = 0.0 if det else parity.GRAD_COND
    if check_world and len(views) == scene.n_views:
        Sw = parity.world_condition(scene, views, ovs, [c["grad_abs"] for c in counts])
        nbad, worst = parity.grad_violations(gpu.grad_verts, gw, Sw, ex, cond)
        assert nbad == 0, f"world gradients: {nbad} components outside tolerance (worst {worst:.3g})"
    if want_attr:
        Sa = sum(c["grad_attr_abs"] for c in counts)
        nbad, worst = parity.grad_violations(gpu.grad_attr, ga, Sa, ex, cond)
        assert nbad == 0, f"attribute gradients: {nbad} outside tolerance (worst {worst:.3g})"
    return gpu, stats, counts


# ---------------------------------------------------------------------------
# projection: snapped positions bit-exact
# ---------------------------------------------------------------------------

def test_project_snap_bitexact(orc):
    import torch

    from paper_2405_02508_gb300 import binding as B

    sc = scenes.head_multiview(n_views=8, H=2048, W=1334, n=64)
    verts = torch.from_numpy(sc.verts).cuda()
    cams = B.cameras_tensor(sc.cams)
    vpix = torch.empty((8, len(sc.verts), 8), dtype=torch.float32, device="cuda")
    B.mer_project(verts, cams, vpix)
    rec = vpix.cpu().numpy()
    ints = rec.view(np.int32)
    for v in range(8):
        scr, snap, flags = orc.project(sc.verts, sc.cams[v])
        np.testing.assert_array_equal(ints[v, :, 6], flags)
        np.testing.assert_array_equal(ints[v, :, 0], snap[:, 0])
        np.testing.assert_array_equal(ints[v, :, 1], snap[:, 1])
        x = snap[:, 0] / 256.0 + rec[v, :, 2]
        np.testing.assert_allclose(x, scr[:, 0], rtol=0, atol=1e-6)
        z = rec[v, :, 4].astype(np.float64) + rec[v, :, 5]
        np.testing.assert_allclose(z, scr[:, 2], rtol=1e-13)


# ---------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------

def test_parity_tiny_icosphere_l2(orc):
    """128^2, 1280 triangles, L2 loss against a target from the perturbed copy."""
    sc = scenes.tiny_icosphere()
    tgt = Scene(sc.name, sc.target_verts, sc.tris, sc.cams, sc.H, sc.W, sc.attr, sc.shading)
    It = orc.render(tgt)[0].image
    Io = orc.render(sc)[0].image
    g = (2.0 * (Io - It))[None].astype(np.float32)
    gpu, stats, counts = run_parity(orc, sc, g, want_attr=True)
    assert stats[0]["covered"] > 5000


@pytest.mark.parametrize("tile,cover_hint", [(8, True), (16, True), (32, True), (16, False)])
def test_parity_intersection_two_spheres(orc, tile, cover_hint):
    """512^2, 2 x 20480 triangles interpenetrating: silhouettes and intersection micro-edges (with and
    without the cover image that lets the backward skip pairs that cannot scatter)."""
    sc = scenes.two_spheres()
    gpu, stats, counts = run_parity(orc, sc, sc.upstream(), tile=tile, cover_hint=cover_hint)
    assert counts[0]["intersection"] > 50


def test_parity_intersections_off(orc):
    sc = scenes.two_spheres(H=256, W=256)
    run_parity(orc, sc, sc.upstream(), terms=1 | 2)


@pytest.mark.parametrize("scene", ["tiny", "two_spheres", "open_sphere"])
def test_parity_exact_crossing_option(orc, scene):
    """The exact-crossing gather option (overhang gradients to the exit edge's endpoints) against the oracle."""
    sc = {"tiny": lambda: scenes.tiny_icosphere(),
          "two_spheres": lambda: scenes.two_spheres(H=256, W=256, subdiv=4),
          "open_sphere": lambda: scenes.open_sphere(H=256, W=256)}[scene]()
    run_parity(orc, sc, sc.upstream(), terms=ALL | 8)


def test_parity_edge_only_and_interior_only(orc):
    sc = scenes.two_spheres(H=256, W=256, subdiv=4)
    run_parity(orc, sc, sc.upstream(), terms=1 | 4)
    run_parity(orc, sc, sc.upstream(), terms=2)


def test_parity_backface_image_and_loss(orc):
    """Back-face image (Supp. B) of an open sphere seen through its hole, with normals and mask: the channel
    equals the oracle's bit for bit; the gradients of N(0,1) upstream and of a pure back-face loss
    (L = sum of the channel: only its edges carry gradient) match the oracle."""
    sc = scenes.open_sphere(H=256, W=256)
    gpu, stats, counts = run_parity(orc, sc, sc.upstream(), want_attr=True)
    bf = gpu.image[..., sc.shading.backface_ch]
    assert 0.1 < bf[gpu.index >= 0].mean() < 0.95
    g = np.zeros((1, sc.H, sc.W, sc.shading.C), np.float32)
    g[..., sc.shading.backface_ch] = 1.0
    gpu2, _, counts2 = run_parity(orc, sc, g)
    assert np.abs(gpu2.grad_verts).max() > 0


@pytest.mark.parametrize("store_bary", [True, False])
def test_parity_head_single_view(orc, store_bary):
    """1024^2, 131k triangles, bilinear texture through interpolated UVs, RGB + mask."""
    sc = scenes.head_single_view()
    run_parity(orc, sc, sc.upstream(), want_attr=True, store_bary=store_bary)


def test_parity_multiview_full_size_sampled_views(orc):
    """32 views at 1334x2048 as the benchmark runs them; the oracle checks 3 sampled views."""
    sc = scenes.head_multiview()
    g = sc.upstream()
    run_parity(orc, sc, g, views=[0, 13, 31], check_world=False)


def test_parity_uneven_items(orc):
    """Items of the uneven batch: smallest, largest and two in between (the flagged-tie share over the four)."""
    items = scenes.uneven_batch(n_items=256)
    T = np.array([len(it.tris) for it in items])
    order = np.argsort(T)
    stats = []
    for i in [order[0], order[len(order) // 3], order[2 * len(order) // 3], order[-1]]:
        it = items[i]
        stats += run_parity(orc, it, it.upstream(), label=f"c5 item {i}", tie_check=False)[1]
    parity.assert_tie_share(stats)


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

def _screen_scene(scr, tris, H, W, C=1, colours=None):
    scr = np.asarray(scr, np.float64)
    colours = np.linspace(0.1, 0.9, len(scr)).astype(np.float32)[:, None] if colours is None else colours
    return scr, np.asarray(tris, np.int32).reshape(-1, 3), H, W, Shading(n_main=1, C=1, bg=[0.25]), colours


def gpu_screen_run(scr, tris, H, W, sh, attr, grads, tile=16, terms=ALL):
    import torch

    from paper_2405_02508_gb300.render import Renderer

    r = Renderer(torch.from_numpy(tris), len(scr), 1, H, W, sh, attr.shape[1], tile=tile)
    r.project_screen(torch.from_numpy(scr[None]).cuda())
    r.rasterize()
    a = torch.from_numpy(attr).cuda()
    r.shade(a, None)
    r.grad_vpix.zero_()
    from paper_2405_02508_gb300 import binding as B

    B.mer_backward(r.vpix, r.tris, r.index, r.image, torch.from_numpy(grads).cuda(), a, None, r.sh, terms,
                   r.grad_vpix, None, r.workspace)
    r.check_status()
    return r.index[0].cpu().numpy(), r.image[0].cpu().numpy(), r.grad_vpix[0].cpu().numpy()


def oracle_screen_run(orc, scr, tris, H, W, sh, attr, grads, terms=ALL):
    s, snap, flags = orc.snap_screen(scr)
    index, tie, _ = orc.rasterize(s, snap, flags, tris, H, W)
    img = orc.shade(s, tris, index, attr, sh)
    gs, _, _, S = orc.backward(s, snap, flags, tris, index, img, grads, attr, sh, mode=terms, want_abs=True)
    return index, tie, img, gs, S


CASES = {
    "ragged_37x53": (_screen_scene([[3.3, 2.1, 0.5], [50.2, 9.7, 0.6], [20.1, 35.2, 0.4],
                                    [10.5, 20.2, 0.7], [45.3, 30.1, 0.3], [30.2, 1.2, 0.5]],
                                   [[0, 1, 2], [3, 4, 5]], 37, 53)),
    "one_pixel": _screen_scene([[-1.0, -1.0, 0.5], [3.0, -1.0, 0.5], [-1.0, 3.0, 0.5]], [[0, 1, 2]], 1, 1),
    "row_1x40": _screen_scene([[2.2, -3.0, 0.5], [30.7, 0.5, 0.5], [11.1, 4.0, 0.5]], [[0, 1, 2]], 1, 40),
    "column_40x1": _screen_scene([[-3.0, 2.2, 0.5], [0.5, 30.7, 0.5], [4.0, 11.1, 0.5]], [[0, 1, 2]], 40, 1),
    "full_screen": _screen_scene([[-100, -100, 0.5], [400, -100, 0.5], [-100, 400, 0.5]], [[0, 1, 2]], 64, 64),
    "all_background": _screen_scene([[-30, -30, 0.5], [-20, -30, 0.5], [-30, -20, 0.5]], [[0, 1, 2]], 32, 32),
    "guard_band": _screen_scene([[-3.0e6, 5.0, 0.5], [40.0, 20.0, 0.5], [10.0, 60.0, 0.5],
                                 [-1.0e5, -1.0e5, 0.5], [2.0e5, 10.0, 0.6], [15.0, 3.0e5, 0.4]],
                                [[0, 1, 2], [3, 4, 5]], 64, 64),
    "behind_camera": _screen_scene([[5.0, 5.0, -0.5], [40.0, 8.0, 0.5], [10.0, 50.0, 0.5],
                                    [6.0, 6.0, 0.5], [50.0, 10.0, 0.5], [12.0, 55.0, 0.5]],
                                   [[0, 1, 2], [3, 4, 5]], 64, 64),
    "degenerate": _screen_scene([[5.0, 5.0, 0.5], [10.0, 10.0, 0.5], [20.0, 20.0, 0.5],
                                 [4.0, 30.0, 0.5], [4.0, 30.0, 0.5], [40.0, 2.0, 0.5]],
                                [[0, 1, 2], [3, 4, 5]], 48, 48),
    "centres_on_edges": _screen_scene([[0.5, 0.5, 0.5], [20.5, 0.5, 0.5], [0.5, 20.5, 0.5], [20.5, 20.5, 0.5],
                                       [10.5, 10.5, 0.6]],
                                      [[0, 1, 4], [1, 3, 4], [3, 2, 4], [2, 0, 4]], 24, 24),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("tile", [8, 16, 32])
def test_edge_cases(orc, case, tile):
    scr, tris, H, W, sh, attr = CASES[case]
    g = np.random.default_rng(1).standard_normal((1, H, W, 1)).astype(np.float32)
    gi, gimg, gg = gpu_screen_run(scr, tris, H, W, sh, attr, g, tile=tile)
    oi, tie, oimg, og, S = oracle_screen_run(orc, scr, tris, H, W, sh, attr, g[0])
    assert np.all((gi == oi) | tie)
    np.testing.assert_allclose(gimg, oimg, rtol=parity.IMG_TOL, atol=parity.IMG_TOL)
    nbad, worst = parity.grad_violations(gg, og, S)
    assert nbad == 0, worst


@pytest.mark.parametrize("shape", [(256, 8192), (8192, 256)])
def test_maximum_image_size(orc, shape):
    """The largest accepted image edge (8192 px), as a strip either way: a soup of 3000 random screen-space
    triangles (sizes from 1 to 300 px, random depths, so overlaps and interpenetrations everywhere) against
    the oracle, every pixel and every vertex."""
    H, W = shape
    rng = np.random.default_rng(8)
    nt = 3000
    c = np.stack([rng.uniform(0, W, nt), rng.uniform(0, H, nt)], axis=1)
    size = np.exp(rng.uniform(np.log(1.0), np.log(300.0), nt))
    pts = c[:, None, :] + rng.normal(0, 1, (nt, 3, 2)) * size[:, None, None]
    z = rng.uniform(0.2, 1.0, (nt, 3))
    scr = np.concatenate([pts, z[..., None]], axis=2).reshape(-1, 3)
    tris = np.arange(3 * nt, dtype=np.int32).reshape(nt, 3)
    sh = Shading(n_main=1, C=1, bg=[0.25])
    attr = rng.uniform(0.1, 0.9, (3 * nt, 1)).astype(np.float32)
    g = rng.standard_normal((1, H, W, 1)).astype(np.float32)
    gi, gimg, gg = gpu_screen_run(scr, tris, H, W, sh, attr, g, tile=32)
    oi, tie, oimg, og, S = oracle_screen_run(orc, scr, tris, H, W, sh, attr, g[0])
    assert np.all((gi == oi) | tie) and (gi >= 0).mean() > 0.5
    same = gi == oi  # flagged near-ties may pick either triangle: their values differ legitimately
    np.testing.assert_allclose(gimg[same], oimg[same], rtol=parity.IMG_TOL, atol=parity.IMG_TOL)
    ex = parity.excluded_vertices(tris, gi, oi)
    nbad, worst = parity.grad_violations(gg, og, S, ex)
    assert nbad == 0, worst


def test_empty_mesh_and_zero_sizes():
    import torch

    from paper_2405_02508_gb300 import binding as B
    from paper_2405_02508_gb300.render import Renderer

    sh = Shading(n_main=0, C=1, mask_ch=0, bg=[0.5])
    r = Renderer(torch.zeros((0, 3), dtype=torch.int32), 0, 2, 20, 30, sh, 1)
    r.project(torch.zeros((0, 3), device="cuda"), B.cameras_tensor(scenes.cameras_on_sphere(2, 3.0, 20, 30, 1)))
    r.rasterize()
    assert torch.all(r.index == -1)
    r.shade(torch.zeros((0, 1), device="cuda"), None)
    assert torch.all(r.image == 0.5)
    r.grad_vpix.zero_()
    B.mer_backward(r.vpix, r.tris, r.index, r.image, torch.ones_like(r.image), torch.zeros((0, 1), device="cuda"),
                   None, r.sh, ALL, r.grad_vpix, None, r.workspace)
    r.check_status()


def test_bin_overflow_reported_and_recovered(orc):
    """A workspace with room for 16 bin entries overflows; the status says so and the exact retry matches."""
    import torch

    from paper_2405_02508_gb300 import binding as B
    from paper_2405_02508_gb300.render import Renderer

    sc = scenes.tiny_icosphere()
    r = Renderer(torch.from_numpy(sc.tris), len(sc.verts), 1, sc.H, sc.W, sc.shading, 3)
    nbytes = B.mer_workspace_size(r.V, r.T, 1, sc.H, sc.W, 16, 16)
    r.workspace = torch.zeros(nbytes // 4 + 64, dtype=torch.float32, device="cuda")
    r.project(torch.from_numpy(sc.verts).cuda(), B.cameras_tensor(sc.cams))
    B.mer_rasterize(r.vpix, r.tris, sc.H, sc.W, 16, r.workspace, r.index)
    code, total = B.mer_sync_status(r.workspace)
    assert code == B.MER_EOVERFLOW and total > 16
    r.rasterize()  # checked path: resizes and redoes
    ov = orc.render(sc)[0]
    assert np.all((r.index[0].cpu().numpy() == ov.index) | ov.tie)


def test_range_errors_reported():
    import torch

    from paper_2405_02508_gb300 import binding as B
    from paper_2405_02508_gb300.render import Renderer

    sh = Shading(n_main=1, C=1, bg=[0.5])
    tris = torch.tensor([[0, 1, 7]], dtype=torch.int32)
    r = Renderer(tris, 3, 1, 16, 16, sh, 1)
    r.project_screen(torch.tensor([[[1.0, 1.0, 0.5], [10.0, 1.0, 0.5], [1.0, 10.0, 0.5]]], dtype=torch.float64).cuda())
    with pytest.raises(B.MerError) as e:
        r.rasterize()
    assert e.value.code == B.MER_ERANGE


def test_invalid_arguments_rejected():
    import torch

    from paper_2405_02508_gb300 import binding as B

    lib = B.lib()
    assert lib.mer_rasterize(None, 3, None, 1, 1, 16, 16, 16, None, 0, None, None, None, None, None) == B.MER_EINVAL
    assert lib.mer_workspace_size(3, 1, 1, 16, 16, 12, 0) == 0  # tile must be 8, 16 or 32
    ws = torch.zeros(1024, device="cuda")
    assert lib.mer_rasterize(None, 3, None, 1, 1, 9000, 16, 16, B._ptr(ws), 4096, None, None, None, None, None) == B.MER_EINVAL


def test_recompute_bary_bitwise_identical():
    """Storing the barycentric image or not changes nothing downstream (the backward re-derives them)."""
    sc = scenes.two_spheres(H=256, W=256, subdiv=4)
    g = sc.upstream()
    a = parity.gpu_run(sc, g, store_bary=True)
    b = parity.gpu_run(sc, g, store_bary=False)
    np.testing.assert_array_equal(a.index, b.index)
    np.testing.assert_array_equal(a.image, b.image)
    # the order of the per-tile FP32 partial sums and of the FP64 atomics may differ between runs, nothing else
    np.testing.assert_allclose(a.grad_verts, b.grad_verts, rtol=1e-5, atol=1e-6 * np.abs(a.grad_verts).max())


def test_rasterize_world_equals_project_then_rasterize():
    """The one-call entry point (world vertices + cameras) gives the same index, depth and records."""
    import torch

    from paper_2405_02508_gb300 import binding as B
    from paper_2405_02508_gb300.render import Renderer

    sc = scenes.head_multiview(n_views=3, H=200, W=160, n=24, tex_size=32)
    verts = torch.from_numpy(sc.verts).cuda()
    cams = B.cameras_tensor(sc.cams)
    r = Renderer(torch.from_numpy(sc.tris), len(sc.verts), 3, 200, 160, sc.shading, 2, sc.tex.shape)
    depth = torch.empty((3, 200, 160), device="cuda")
    r.project(verts, cams)
    r.rasterize(depth)
    idx0, d0, v0 = r.index.clone(), depth.clone(), r.vpix.clone()
    r.index.fill_(-7)
    r.vpix.zero_()
    B.mer_rasterize_world(verts, r.tris, cams, 200, 160, r.tile, r.workspace, r.index, r.vpix, depth)
    r.check_status()
    assert torch.equal(r.index, idx0) and torch.equal(depth, d0)
    assert torch.equal(r.vpix.view(torch.int32), v0.view(torch.int32))  # records hold integer fields


def test_recompute_option_peak_memory():
    """Head-scale single view (1024^2, 131k triangles) through the autograd function: storing the barycentric
    image costs its 8 B per pixel of peak device memory, recomputing it in the backward does not, and the
    gradients agree."""
    import torch

    from paper_2405_02508_gb300 import binding as B
    from paper_2405_02508_gb300.render import MerRender, Renderer

    sc = scenes.head_single_view()
    tex = torch.from_numpy(sc.tex).cuda()
    cams = B.cameras_tensor(sc.cams)
    g = torch.from_numpy(sc.upstream()).cuda()
    r = Renderer(torch.from_numpy(sc.tris), len(sc.verts), 1, sc.H, sc.W, sc.shading, 2, tex.shape)
    peak, grads = {}, {}
    for recompute in (True, False, True):
        verts = torch.from_numpy(sc.verts).cuda().requires_grad_(True)
        attr = torch.from_numpy(sc.attr).cuda().requires_grad_(True)
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()
        base = torch.cuda.memory_allocated()
        img = MerRender.apply(verts, attr, tex, cams, r, recompute)
        (img * g).sum().backward()
        torch.cuda.synchronize()
        peak[recompute] = torch.cuda.max_memory_allocated() - base
        grads[recompute] = verts.grad.cpu().numpy()
    print(f"peak extra memory: recompute {peak[True] / 2**20:.1f} MiB, stored bary {peak[False] / 2**20:.1f} MiB")
    assert peak[False] - peak[True] >= 8 * sc.H * sc.W
    np.testing.assert_allclose(grads[True], grads[False], rtol=1e-5, atol=1e-6 * np.abs(grads[False]).max())


def test_modular_entry_points_sum_to_fused(orc):
    """mer_edge_grad_backward + mer_interpolate_backward reproduce the fused backward (plain interpolation)."""
    import torch

    from paper_2405_02508_gb300 import binding as B
    from paper_2405_02508_gb300.render import Renderer

    sc = scenes.tiny_icosphere()
    g = sc.upstream()
    fused = parity.gpu_run(sc, g)
    r = Renderer(torch.from_numpy(sc.tris), len(sc.verts), 1, sc.H, sc.W, sc.shading, 3)
    cams = B.cameras_tensor(sc.cams)
    attr = torch.from_numpy(sc.attr).cuda()
    r.forward(torch.from_numpy(sc.verts).cuda(), cams, attr)
    gt = torch.from_numpy(g).cuda()
    gv = torch.zeros_like(r.grad_vpix)
    B.mer_edge_grad_backward(r.image, gt, r.index, r.vpix, r.tris, True, gv, r.workspace)
    ga = torch.zeros_like(attr)
    B.mer_interpolate_backward(attr, r.tris, r.vpix, r.index, gt, ga, gv, r.workspace)
    r.check_status()
    np.testing.assert_allclose(gv.cpu().numpy(), fused.grad_vpix, rtol=1e-4, atol=1e-6)


def test_autograd_function_matches_renderer():
    import torch

    from paper_2405_02508_gb300 import binding as B
    from paper_2405_02508_gb300.render import MerRender, Renderer

    sc = scenes.head_single_view(H=256, W=256, n=32, tex_size=128)
    g = torch.from_numpy(sc.upstream()).cuda()
    ref = parity.gpu_run(sc, sc.upstream(), want_attr=True)
    for recompute in (True, False):
        r = Renderer(torch.from_numpy(sc.tris), len(sc.verts), 1, sc.H, sc.W, sc.shading, 2, sc.tex.shape)
        verts = torch.from_numpy(sc.verts).cuda().requires_grad_(True)
        attr = torch.from_numpy(sc.attr).cuda().requires_grad_(True)
        img = MerRender.apply(verts, attr, torch.from_numpy(sc.tex).cuda(), B.cameras_tensor(sc.cams), r, recompute)
        (img * g).sum().backward()
        # same kernels as the reference run; only the order of the FP32 attribute atomics differs, so the
        # bound is relative to the largest component (cancelling sums differ by summation-order noise)
        np.testing.assert_allclose(verts.grad.cpu().numpy(), ref.grad_verts, rtol=1e-4,
                                   atol=1e-6 * np.abs(ref.grad_verts).max())
        np.testing.assert_allclose(attr.grad.cpu().numpy(), ref.grad_attr, rtol=1e-4,
                                   atol=1e-5 * np.abs(ref.grad_attr).max())
