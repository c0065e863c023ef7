"""The cover image: what the rasterizers record about the triangles covering each pixel centre, and the
backward pass that uses it to skip pixel pairs that cannot scatter.

A pair (p, q) with triangles t_p != t_q scatters into p's fragment only if t_q also covers p's centre
(Sec. 4.3: p lies on top of t_q, or the two intersect).  The cover image must therefore never rule out a pair
for which the oracle's exact coverage predicate says that t_q covers p (no false negatives); the gradients
with and without it must agree and both match the oracle.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_2405_02508_gb300 import scenes

from . import parity

pytestmark = pytest.mark.gpu

SAME_2, OTHER_1, WINNER_BACK, BORDER_L, BORDER_R, BORDER_T, BORDER_B = 1, 2, 4, 8, 16, 32, 64


@pytest.fixture(scope="module")
def orc():
    import oracle

    oracle.build()
    return oracle


def _may_scatter(cp, cq, border_bit):
    """The backward's test for a pair whose neighbour q is covered: can q's triangle cover p's centre?  (Across
    the border of p's bin tile the back-facing counts may leave out q's triangle when it is back-facing.)"""
    same = ((cp ^ cq) & WINNER_BACK) == 0
    need = np.where(same, cp & SAME_2, cp & OTHER_1) != 0
    return need | (((cp & border_bit) != 0) & ((cq & WINNER_BACK) != 0))


def check_cover(orc, index, cover, snap, flags, tris, tile):
    """Asserts the cover image's bits for one view; returns (pairs with both pixels covered, pairs ruled
    out by the cover image)."""
    H, W = index.shape
    ys, xs = np.mgrid[0:H, 0:W]
    # border bits: first / last column and row of the pixel's bin tile
    np.testing.assert_array_equal((cover & BORDER_L) != 0, (xs % tile) == 0)
    np.testing.assert_array_equal((cover & BORDER_R) != 0, (xs % tile) == tile - 1)
    np.testing.assert_array_equal((cover & BORDER_T) != 0, (ys % tile) == 0)
    np.testing.assert_array_equal((cover & BORDER_B) != 0, (ys % tile) == tile - 1)
    covered = index >= 0
    assert not (cover[~covered] & (SAME_2 | OTHER_1 | WINNER_BACK)).any()
    # the winner's facing: positive snapped area (clockwise on screen, y down) is back-facing
    t = index[covered]
    X = snap[tris[t], 0].astype(np.int64)
    Y = snap[tris[t], 1].astype(np.int64)
    a2 = (X[:, 1] - X[:, 0]) * (Y[:, 2] - Y[:, 0]) - (Y[:, 1] - Y[:, 0]) * (X[:, 2] - X[:, 0])
    back = (cover[covered] & WINNER_BACK) != 0
    np.testing.assert_array_equal(back, a2 > 0)
    n_pairs = n_skipped = 0
    for horizontal in (True, False):
        for sgn in (1, -1):  # p's neighbour to the right / below, then to the left / above
            if horizontal:
                sp = (slice(None), slice(0, W - 1)) if sgn > 0 else (slice(None), slice(1, W))
                sq = (slice(None), slice(1, W)) if sgn > 0 else (slice(None), slice(0, W - 1))
            else:
                sp = (slice(0, H - 1), slice(None)) if sgn > 0 else (slice(1, H), slice(None))
                sq = (slice(1, H), slice(None)) if sgn > 0 else (slice(0, H - 1), slice(None))
            ip, iq = index[sp], index[sq]
            sel = (ip >= 0) & (iq >= 0) & (ip != iq)
            border = (BORDER_R if sgn > 0 else BORDER_L) if horizontal else (BORDER_B if sgn > 0 else BORDER_T)
            may = _may_scatter(cover[sp][sel].astype(np.int64), cover[sq][sel].astype(np.int64), border)
            py, px = ys[sp][sel], xs[sp][sel]
            tq = iq[sel]
            n_pairs += int(sel.sum())
            n_skipped += int((~may).sum())
            for k in np.nonzero(~may)[0]:
                assert not orc.covers_pixel(snap, flags, tris, int(tq[k]), int(px[k]), int(py[k])), (
                    f"pair at ({px[k]}, {py[k]}) ruled out although triangle {tq[k]} covers the pixel centre")
    return n_pairs, n_skipped


def _per_view(orc, sc, tile):
    import torch

    from paper_2405_02508_gb300 import binding as B
    from paper_2405_02508_gb300.render import Renderer

    r = Renderer(torch.from_numpy(sc.tris), len(sc.verts), sc.n_views, sc.H, sc.W, sc.shading, sc.attr.shape[1],
                 None if sc.tex is None else sc.tex.shape, tile=tile)
    r.project(torch.from_numpy(sc.verts).cuda(), B.cameras_tensor(sc.cams))
    r.rasterize()
    return r.index.cpu().numpy(), r.cover.cpu().numpy()


@pytest.mark.parametrize("tile", [8, 16, 32])
@pytest.mark.parametrize("name", ["two_spheres", "open_sphere", "tiny"])
def test_cover_rules_out_only_pairs_that_cannot_scatter(orc, name, tile):
    sc = {"two_spheres": lambda: scenes.two_spheres(H=256, W=224), "open_sphere": lambda: scenes.open_sphere(),
          "tiny": lambda: scenes.tiny_icosphere()}[name]()
    index, cover = _per_view(orc, sc, tile)
    ov = orc.render(sc)[0]
    n_pairs, n_skipped = check_cover(orc, index[0], cover[0], ov.snap, ov.flags, sc.tris, tile)
    assert n_pairs > 500
    # adjacent triangles of a closed surface are the common case: most pairs need no classification, except
    # where two front surfaces overlap (the two spheres interpenetrate over much of their projected disks)
    assert n_skipped > {"two_spheres": 0.3, "open_sphere": 0.5, "tiny": 0.5}[name] * n_pairs, (n_pairs, n_skipped)


@pytest.mark.parametrize("tile", [16, 32, 64])
def test_batch_cover_rules_out_only_pairs_that_cannot_scatter(orc, tile):
    import torch

    from paper_2405_02508_gb300.batch import BatchRenderer

    sc = scenes.head_multiview(n_views=3, H=300, W=260, n=40, tex_size=256)
    tex = torch.from_numpy(sc.tex).cuda()
    br = BatchRenderer([(sc.verts, sc.tris)], [(0, v, sc.H, sc.W) for v in range(3)], sc.cams, sc.shading,
                       sc.attr.shape[1], tex, tile=tile)
    br.prepare(torch.from_numpy(sc.verts).cuda(), torch.from_numpy(sc.attr).cuda(), tex)
    index = br.index.cpu().numpy().reshape(3, sc.H, sc.W)
    cover = br.cover.cpu().numpy().reshape(3, sc.H, sc.W)
    ovs = orc.render(sc)
    for v in range(3):
        n_pairs, n_skipped = check_cover(orc, index[v], cover[v], ovs[v].snap, ovs[v].flags, sc.tris, tile)
        assert n_skipped > 0.5 * n_pairs


@pytest.mark.parametrize("tile", [16, 64])
def test_batch_backward_with_and_without_cover(tile):
    """The batched backward gives the same gradients with the cover image as without it (up to the
    summation order of the per-tile sums)."""
    import torch

    from paper_2405_02508_gb300.batch import BatchRenderer

    sc = scenes.two_spheres(H=320, W=288)
    g = torch.from_numpy(sc.upstream()).cuda().reshape(-1, sc.shading.C)
    verts = torch.from_numpy(sc.verts).cuda()
    attr = torch.from_numpy(sc.attr).cuda()
    out = {}
    for hint in (True, False):
        br = BatchRenderer([(sc.verts, sc.tris)], [(0, 0, sc.H, sc.W)], sc.cams, sc.shading, sc.attr.shape[1], None,
                           tile=tile, cover_hint=hint)
        br.prepare(verts, attr)
        br.backward(g, attr)
        br.check()
        out[hint] = br.grad_vpix.cpu().numpy()
    ref = out[False]
    np.testing.assert_allclose(out[True], ref, rtol=1e-5, atol=1e-6 * np.abs(ref).max())


def test_parity_open_sphere_with_cover(orc):
    """Back faces seen through an opening: per-view backward with the cover image against the oracle."""
    import torch  # noqa: F401

    sc = scenes.open_sphere()
    g = sc.upstream()
    gpu = parity.gpu_run(sc, g, tile=16)
    ov = orc.render(sc)
    gs, gw, counts, _ = orc.backward_scene(sc, ov, [g[0]])
    parity.compare_view(gpu, 0, ov[0], gs[0], sc.tris, S=counts[0]["grad_abs"])
