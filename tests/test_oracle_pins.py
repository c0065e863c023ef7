"""Pins of the FP64 oracle against ground truth that is not the oracle itself.

Each test names what it pins.  P1..P8 follow the pin list of the design notes:
exact discrete identities (ramp, translation invariance), closed-form boundary
gradients (single triangle, intersection line), box-filtered finite
differences computed by exact polygon clipping, frozen-visibility finite
differences of the interior term, special cases, and brute-force raster
properties (watertightness, closed-mesh double coverage, exact interior /
exterior, depth order by an independent plane fit).
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2405_02508_gb300 import scenes
from paper_2405_02508_gb300.scenes import Shading

from . import geom

EDGE, INTERIOR, INTERSECT = 1, 2, 4
ALL = EDGE | INTERIOR | INTERSECT


def flat_scene(orc, scr, tris, H, W, colours, bg):
    """Screen-space scene, one channel, per-vertex colour."""
    scr, snap, flags = orc.snap_screen(np.asarray(scr, dtype=np.float64))
    tris = np.asarray(tris, dtype=np.int32)
    index, tie, _ = orc.rasterize(scr, snap, flags, tris, H, W)
    attr = np.asarray(colours, dtype=np.float32).reshape(-1, 1)
    sh = Shading(n_main=1, C=1, bg=[bg])
    image = orc.shade(scr, tris, index, attr, sh)
    return scr, snap, flags, tris, index, tie, attr, sh, image


# ---------------------------------------------------------------------------
# projection
# ---------------------------------------------------------------------------

def test_projection_matches_homogeneous_pinhole(orc):
    """Vertex transform: same x_s, y_s, zeta as K [R|t] with a homogeneous divide; snap = rint(256 x_s)."""
    rng = np.random.default_rng(11)
    verts = rng.uniform(-1.0, 1.0, (500, 3)).astype(np.float32)
    for cam in scenes.cameras_on_sphere(4, 3.0, 300, 200, seed=12):
        scr, snap, flags = orc.project(verts, cam)
        ref = geom.project_homogeneous(verts, cam)
        assert np.all(flags == 3)
        np.testing.assert_allclose(scr, ref, rtol=1e-12, atol=1e-9)
        np.testing.assert_array_equal(snap, np.rint(scr[:, :2] * 256.0).astype(np.int64))


def test_projection_orientation_and_near_plane(orc):
    """World +x lands right of centre and +y above it for a camera on +z; points behind are invalid."""
    cam = scenes.look_at_camera((0.0, 0.0, 3.0), 100, 100)
    v = np.array([[0, 0, 0], [0.5, 0, 0], [0, 0.5, 0], [0, 0, 3.5], [0, 0, 2.95]], np.float32)
    scr, snap, flags = orc.project(v, cam)
    assert scr[0, 0] == pytest.approx(50.0) and scr[0, 1] == pytest.approx(50.0)
    assert scr[0, 2] == pytest.approx(1.0 / 3.0)
    assert scr[1, 0] > 50.0 and scr[2, 1] < 50.0
    assert flags[3] == 0 and flags[4] == 0  # behind the camera / in front of the near plane 0.1
    assert np.all(flags[:3] == 3)


# ---------------------------------------------------------------------------
# P8 raster: brute-force properties
# ---------------------------------------------------------------------------

def _coverage_counts(orc, snap, flags, tris, H, W):
    cnt = np.zeros((H, W), np.int32)
    who = np.full((H, W), -1, np.int32)
    for t in range(len(tris)):
        for y in range(H):
            for x in range(W):
                if orc.covers_pixel(snap, flags, tris, t, x, y):
                    cnt[y, x] += 1
                    who[y, x] = t
    return cnt, who


def _jittered_grid(nx, ny, W, H, rng, snap_to_centres=False):
    xs = np.linspace(0.0, W, nx + 1)
    ys = np.linspace(0.0, H, ny + 1)
    P = np.array([[x, y] for y in ys for x in xs])
    inner = (P[:, 0] > 0) & (P[:, 0] < W) & (P[:, 1] > 0) & (P[:, 1] < H)
    P[inner] += rng.uniform(-0.35, 0.35, (inner.sum(), 2)) * (W / nx)
    if snap_to_centres:  # put interior vertices exactly on pixel centres -> edges through centres
        P[inner] = np.floor(P[inner]) + 0.5
    T = []
    for j in range(ny):
        for i in range(nx):
            a = j * (nx + 1) + i
            b, c, d = a + 1, a + nx + 1, a + nx + 2
            if (i + j) % 2:
                T += [[a, b, d], [a, d, c]]
            else:
                T += [[a, b, c], [b, d, c]]
    T = np.array(T, np.int32)
    flip = rng.uniform(size=len(T)) < 0.5  # mixed windings
    T[flip] = T[flip][:, ::-1]
    scr = np.concatenate([P, np.full((len(P), 1), 0.5)], axis=1)
    return scr, T


@pytest.mark.parametrize("snap_centres", [False, True])
def test_p8_watertight_planar_grid(orc, snap_centres):
    """A triangulated grid over the whole image covers every pixel centre exactly once."""
    rng = np.random.default_rng(21 + snap_centres)
    H, W = 20, 24
    scr, T = _jittered_grid(4, 3, W, H, rng, snap_centres)
    scr, snap, flags = orc.snap_screen(scr)
    cnt, who = _coverage_counts(orc, snap, flags, T, H, W)
    assert np.all(cnt == 1)
    index, tie, _ = orc.rasterize(scr, snap, flags, T, H, W)
    np.testing.assert_array_equal(index, who)


def test_p8_watertight_axis_aligned_edges_through_centres(orc):
    """Horizontal and vertical edges exactly through pixel centres: still exactly one owner per pixel."""
    H, W = 20, 24
    xs = np.array([0.0, 3.5, 7.5, 12.5, 18.5, 24.0])
    ys = np.array([0.0, 4.5, 9.5, 13.5, 20.0])
    P = np.array([[x, y] for y in ys for x in xs])
    nx = len(xs) - 1
    T = []
    for j in range(len(ys) - 1):
        for i in range(nx):
            a = j * (nx + 1) + i
            b, c, d = a + 1, a + nx + 1, a + nx + 2
            T += [[a, b, d], [a, d, c]] if (i + j) % 2 else [[a, b, c], [b, d, c]]
    T = np.array(T, np.int32)
    T[1::3] = T[1::3][:, ::-1]
    scr, snap, flags = orc.snap_screen(np.concatenate([P, np.full((len(P), 1), 0.5)], axis=1))
    cnt, who = _coverage_counts(orc, snap, flags, T, H, W)
    assert np.all(cnt == 1)


def test_p8_closed_mesh_double_coverage(orc):
    """A closed convex mesh seen from outside covers each pixel centre 0 or 2 times, 2 well inside."""
    P, F = scenes.icosphere(2)
    cam = scenes.look_at_camera((0.0, 0.0, 3.0), 28, 30)
    scr, snap, flags = orc.project(P.astype(np.float32), cam)
    cnt, _ = _coverage_counts(orc, snap, flags, F, 28, 30)
    assert set(np.unique(cnt).tolist()) <= {0, 2}
    # the sphere's silhouette radius in pixels: fy * r / sqrt(d^2 - r^2) (inscribed icosphere is a bit smaller)
    fy = float(cam["fy"])
    r_sil = fy / math.sqrt(8.0)
    yy, xx = np.mgrid[0:28, 0:30] + 0.5
    rad = np.hypot(xx - 15.0, yy - 14.0)
    assert np.all(cnt[rad < 0.85 * r_sil] == 2)
    assert np.all(cnt[rad > r_sil + 0.5] == 0)


def test_p8_exact_interior_exterior_and_depth_order(orc):
    """Centres strictly inside (exact rational barycentrics) are covered, strictly outside are not;
    the winner is the triangle with the largest plane-fitted zeta (away from near-ties)."""
    rng = np.random.default_rng(31)
    H, W = 24, 28
    nt = 12
    V = rng.uniform(-4, 32, (3 * nt, 2))
    z = np.repeat(rng.uniform(0.2, 0.9, nt), 3) * rng.uniform(0.95, 1.05, 3 * nt)
    scr = np.concatenate([V, z[:, None]], axis=1)
    T = np.arange(3 * nt, dtype=np.int32).reshape(nt, 3)
    scr, snap, flags = orc.snap_screen(scr)
    index, tie, _ = orc.rasterize(scr, snap, flags, T, H, W)
    for t in range(nt):
        Xs = [Fraction(int(snap[v, 0]), 256) for v in T[t]]
        Ys = [Fraction(int(snap[v, 1]), 256) for v in T[t]]
        det = (Xs[1] - Xs[0]) * (Ys[2] - Ys[0]) - (Ys[1] - Ys[0]) * (Xs[2] - Xs[0])
        if det == 0:
            continue
        # plane through (X/256, Y/256, zeta) by least squares on 3 points (exact fit)
        A = np.array([[float(Xs[i]), float(Ys[i]), 1.0] for i in range(3)])
        plane = np.linalg.solve(A, scr[T[t], 2])
        for y in range(H):
            for x in range(W):
                px, py = Fraction(2 * x + 1, 2), Fraction(2 * y + 1, 2)
                l1 = ((px - Xs[0]) * (Ys[2] - Ys[0]) - (py - Ys[0]) * (Xs[2] - Xs[0])) / det
                l2 = ((Xs[1] - Xs[0]) * (py - Ys[0]) - (Ys[1] - Ys[0]) * (px - Xs[0])) / det
                l0 = 1 - l1 - l2
                inside = l0 > 0 and l1 > 0 and l2 > 0
                outside = l0 < 0 or l1 < 0 or l2 < 0
                cov = orc.covers_pixel(snap, flags, T, t, x, y)
                if inside:
                    assert cov
                if outside:
                    assert not cov
                if cov and not tie[y, x]:
                    w = index[y, x]
                    zt = plane @ np.array([x + 0.5, y + 0.5, 1.0])
                    Aw = np.array([[snap[v, 0] / 256.0, snap[v, 1] / 256.0, 1.0] for v in T[w]])
                    zw = np.linalg.solve(Aw, scr[T[w], 2]) @ np.array([x + 0.5, y + 0.5, 1.0])
                    assert zw >= zt * (1 - 1e-9)


def test_p8_tie_flags_and_tie_break(orc):
    """Coplanar duplicates are flagged and resolved to the lower id; a 1e-7 relative gap is flagged,
    a 1e-3 gap is not."""
    base = np.array([[2.0, 2.0], [30.0, 4.0], [10.0, 28.0]])
    for gap, flagged in [(0.0, True), (1e-7, True), (1e-3, False)]:
        scr = np.concatenate([np.concatenate([base, base]),
                              np.array([[0.5]] * 3 + [[0.5 * (1 + gap)]] * 3)], axis=1)
        T = np.array([[3, 4, 5], [0, 1, 2]], np.int32)  # the nearer copy has the higher id when gap > 0
        s, snap, flags = orc.snap_screen(scr)
        index, tie, _ = orc.rasterize(s, snap, flags, T, 32, 32)
        cov = index >= 0
        assert cov.sum() > 100
        assert np.all(tie[cov] == flagged)
        assert np.all(index[cov] == 0)  # gap 0: lower id wins; gap > 0: id 0 is nearer


# ---------------------------------------------------------------------------
# P1 exact ramp identity
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("axis", [0, 1])
def test_p1_ramp_identity_single_triangle(orc, axis):
    """L = sum_p coord_p I_p: the x (y) vertex gradients sum to (c - bg) x #covered exactly."""
    H, W = 40, 48
    c, bg = 0.75, 0.25
    s = flat_scene(orc, [[5.3, 4.1, 0.5], [41.7, 9.9, 0.5], [17.2, 35.6, 0.5]], [[0, 1, 2]], H, W, [c] * 3, bg)
    scr, snap, flags, tris, index, tie, attr, sh, image = s
    yy, xx = np.mgrid[0:H, 0:W] + 0.5
    g = (xx if axis == 0 else yy)[..., None].astype(np.float32)
    gs, _, cnt = orc.backward(scr, snap, flags, tris, index, image, g, attr, sh, mode=ALL)
    ncov = int((index >= 0).sum())
    assert gs[:, axis].sum() == pytest.approx((c - bg) * ncov, rel=1e-12, abs=1e-9)
    assert abs(gs[:, 1 - axis].sum()) < 1e-9 * ncov
    assert np.abs(gs[:, 2]).max() < 1e-9  # overhang: no zeta component; flat colour: no interior term
    assert cnt["overhang"] == cnt["differing"]


@pytest.mark.parametrize("case", ["occlusion", "intersection"])
def test_p1_ramp_identity_two_triangles(orc, case):
    """Same identity with two flat triangles: one over the other (overhang between triangles) or
    interpenetrating (intersection pairs; the two Eq. 12 terms must sum to the full shift)."""
    H, W = 44, 52
    if case == "occlusion":
        # the front triangle lies inside the back one: no outline crossings, hence no pair that
        # the classification calls adjacent although the colours differ
        scr = [[10.3, 9.7, 0.6], [34.6, 11.8, 0.6], [13.9, 29.6, 0.6],
               [1.2, 1.7, 0.3], [50.3, 2.9, 0.3], [3.1, 42.6, 0.3]]
    else:
        # triangle 0 lies inside triangle 1's outline and crosses its plane along a diagonal line
        P0 = [[10.3, 9.7], [34.6, 11.8], [13.9, 29.6]]
        P1 = [[1.2, 1.7], [50.3, 2.9], [3.1, 42.6]]
        scr = [[x, y, 0.45 + 0.01 * (y - 15.0) + 0.004 * (x - 20.0)] for x, y in P0] + \
              [[x, y, 0.45 + 0.01 * (x - 20.0) - 0.003 * (y - 15.0)] for x, y in P1]
    c1, c2, bg = 0.875, 0.375, 0.125
    s = flat_scene(orc, scr, [[0, 1, 2], [3, 4, 5]], H, W, [c1] * 3 + [c2] * 3, bg)
    scr, snap, flags, tris, index, tie, attr, sh, image = s
    yy, xx = np.mgrid[0:H, 0:W] + 0.5
    for axis, coord in ((0, xx), (1, yy)):
        g = coord[..., None].astype(np.float32)
        gs, _, cnt = orc.backward(scr, snap, flags, tris, index, image, g, attr, sh, mode=ALL)
        expect = float((image[..., 0] - bg).sum())
        assert gs[:, axis].sum() == pytest.approx(expect, rel=1e-11)
        assert cnt["adjacent"] == 0
        if case == "occlusion":
            # per triangle: the front one carries (c1 - c2) x its pixels, the back one (c2 - bg) x the
            # pixels inside its outline (visible or hidden), so the foreground choice is pinned too
            n_front = int((index == 0).sum())
            n_back_outline = int((index >= 0).sum())
            assert gs[:3, axis].sum() == pytest.approx((c1 - c2) * n_front, rel=1e-11)
            assert gs[3:, axis].sum() == pytest.approx((c2 - bg) * n_back_outline, rel=1e-11)
    if case == "intersection":
        assert cnt["intersection"] > 10
    else:
        assert cnt["intersection"] == 0 and cnt["overhang"] > cnt["differing"] // 2


# ---------------------------------------------------------------------------
# P2 closed-form boundary gradient of a single flat triangle
# ---------------------------------------------------------------------------

def _area_gradient(P2):
    """d(area)/d(v_i) for a triangle [3,2]: half the outward normal of the opposite edge times its length."""
    g = np.zeros((3, 2))
    area2 = (P2[1, 0] - P2[0, 0]) * (P2[2, 1] - P2[0, 1]) - (P2[1, 1] - P2[0, 1]) * (P2[2, 0] - P2[0, 0])
    s = 1.0 if area2 > 0 else -1.0
    for i in range(3):
        j, k = (i + 1) % 3, (i + 2) % 3
        e = P2[k] - P2[j]
        g[i] = 0.5 * s * np.array([-e[1], e[0]])
    return g


def test_p2_closed_form_boundary_gradient_converges(orc):
    """g = 1: dL/dv_i -> (c - bg) d(area)/d(v_i); relative error falls ~1/N and is < 1 % at N = 1024."""
    c, bg = 0.75, 0.25
    unit = np.array([[0.113, 0.097], [0.871, 0.233], [0.352, 0.904]])
    errs = []
    Ns = [64, 128, 256, 512, 1024]
    for N in Ns:
        P2 = unit * N
        scr = np.concatenate([P2, np.full((3, 1), 0.5)], axis=1)
        s = flat_scene(orc, scr, [[0, 2, 1]], N, N, [c] * 3, bg)
        scr, snap, flags, tris, index, tie, attr, sh, image = s
        g = np.ones((N, N, 1), np.float32)
        gs, _, _ = orc.backward(scr, snap, flags, tris, index, image, g, attr, sh, mode=ALL)
        ref = (c - bg) * _area_gradient(P2)
        errs.append(np.linalg.norm(gs[:, :2] - ref) / np.linalg.norm(ref))
    assert errs[-1] < 0.01
    assert errs[-1] < errs[0] / 4  # converges roughly like 1/N
    assert all(e2 < e1 * 1.3 for e1, e2 in zip(errs, errs[1:]))


# ---------------------------------------------------------------------------
# P3 translation invariance, full pipeline with projection
# ---------------------------------------------------------------------------

def _interior_dIdx(scr, tris, index, attr_rgb):
    """Per-pixel screen derivative d(attr)/dP_x of perspective-correct interpolation (matrix inverse)."""
    H, W = index.shape
    out = np.zeros((H, W, attr_rgb.shape[1]))
    for y in range(H):
        for x in range(W):
            t = index[y, x]
            if t < 0:
                continue
            vi = tris[t]
            P2 = scr[vi, :2]
            z = scr[vi, 2]
            Minv, grad = geom.lambda_gradients(P2)
            lam = Minv @ np.array([x + 0.5, y + 0.5, 1.0])
            s = lam @ z
            num = (lam * z) @ attr_rgb[vi]
            ds = grad[:, 0] @ z
            dnum = (grad[:, 0] * z) @ attr_rgb[vi]
            out[y, x] = (dnum * s - num * ds) / (s * s)
    return out


def test_p3_translation_invariance_world_shift(orc):
    """Image-space shift of the whole mesh (dV = R^T (Z/fx, 0, 0) dt): summed vertex gradient equals
    sum over horizontal overhang/intersection pairs of dL/dp plus sum_p g . (-dI/dx) of the interior."""
    sc = scenes.tiny_icosphere(H=48, W=56)
    sc.cams = scenes.cameras_on_sphere(1, 3.0, sc.H, sc.W, seed=17)  # oblique: R is not symmetric
    r = orc.render_view(sc.verts, sc.tris, sc.cams[0], sc.H, sc.W, sc.attr, sc.shading)
    g = np.random.default_rng(5).standard_normal(r.image.shape).astype(np.float32)
    gs, _, cnt = orc.backward(r.scr, r.snap, r.flags, sc.tris, r.index, r.image, g, sc.attr, sc.shading, mode=ALL)
    gw = orc.project_backward(sc.verts, sc.cams[0], gs)
    cam = sc.cams[0]
    R = np.asarray(cam["R"]).reshape(3, 3)
    Zc = (sc.verts.astype(np.float64) @ R.T + np.asarray(cam["t"]))[:, 2]
    dV = (Zc / float(cam["fx"]))[:, None] * R[0][None, :]  # R^T (Z/fx, 0, 0)
    lhs = float((gw * dV).sum())
    # right-hand side from images, index and independent derivatives
    H, W = r.index.shape
    edge = 0.0
    for y in range(H):
        for x in range(W - 1):
            ta, tb = r.index[y, x], r.index[y, x + 1]
            if ta == tb:
                continue
            if ta >= 0 and tb >= 0:
                b_in_a = orc.covers_pixel(r.snap, r.flags, sc.tris, ta, x + 1, y)
                a_in_b = orc.covers_pixel(r.snap, r.flags, sc.tris, tb, x, y)
                if not b_in_a and not a_in_b:
                    continue
            edge += float(0.5 * (g[y, x].astype(np.float64) + g[y, x + 1]) @ (r.image[y, x] - r.image[y, x + 1]))
    dIdx = _interior_dIdx(r.scr, sc.tris, r.index, sc.attr.astype(np.float64))
    interior = -float((g * dIdx).sum())
    assert lhs == pytest.approx(edge + interior, rel=1e-9, abs=1e-9)
    assert abs(interior) > 1e-3 and abs(edge) > 1e-3


# ---------------------------------------------------------------------------
# P4 two-triangle intersection line
# ---------------------------------------------------------------------------

def _intersection_scene(orc, N, vertical_line):
    """Two large flat-coloured triangles (edges outside the image) crossing along one line."""
    big = np.array([[-2.0, -2.0], [5.0, -1.5], [-1.5, 5.0]])
    P1 = big * N
    P2 = (big[[0, 2, 1]] + np.array([0.05, -0.07])) * N
    if vertical_line:
        # zeta_1 - zeta_2 depends on x only: the line is x = 0.43 N
        z = lambda P: 1.0 + 0.2 * (P[:, 0] / N - 0.43)  # noqa: E731
        z2 = lambda P: np.full(len(P), 1.0)  # noqa: E731
    else:
        z = lambda P: 1.0 + 0.2 * (P[:, 0] / N - 0.43) + 0.13 * (P[:, 1] / N - 0.51)  # noqa: E731
        z2 = lambda P: 1.0 + 0.05 * (P[:, 1] / N - 0.51) - 0.06 * (P[:, 0] / N - 0.43)  # noqa: E731
    scr = np.concatenate([np.concatenate([P1, z(P1)[:, None]], 1), np.concatenate([P2, z2(P2)[:, None]], 1)])
    c1, c2, bg = 0.875, 0.25, 0.0
    s = flat_scene(orc, scr, [[0, 1, 2], [3, 4, 5]], N, N, [c1] * 3 + [c2] * 3, bg)
    # f(P) = zeta_1(P) - zeta_2(P) = alpha . P + beta, by plane fits through each triangle
    A1 = np.concatenate([P1, np.ones((3, 1))], 1)
    A2 = np.concatenate([P2, np.ones((3, 1))], 1)
    pl1 = np.linalg.solve(A1, scr[:3, 2])
    pl2 = np.linalg.solve(A2, scr[3:, 2])
    return s, c1 - c2, pl1, pl2


def _line_length_in_square(alpha, beta, N):
    """Length of {alpha . P + beta = 0} inside [0, N]^2."""
    pts = []
    for xc in (0.0, N):
        if abs(alpha[1]) > 1e-300:
            y = -(alpha[0] * xc + beta) / alpha[1]
            if 0 <= y <= N:
                pts.append((xc, y))
    for yc in (0.0, N):
        if abs(alpha[0]) > 1e-300:
            x = -(alpha[1] * yc + beta) / alpha[0]
            if 0 <= x <= N:
                pts.append((x, yc))
    pts = sorted(set(pts))
    assert len(pts) >= 2
    return math.dist(pts[0], pts[-1])


@pytest.mark.parametrize("vertical_line", [True, False])
def test_p4_intersection_in_image_shift_converges(orc, vertical_line):
    """Shifting triangle 1 along x by d: dL/dd = -(c1 - c2) a1_x / |grad f| * length (g = 1).
    The micro-edge estimate (intersection pairs only; triangle edges lie outside) reproduces it."""
    errs = []
    for N in (32, 64, 128):
        s, jump, pl1, pl2 = _intersection_scene(orc, N, vertical_line)
        scr, snap, flags, tris, index, tie, attr, sh, image = s
        g = np.ones((N, N, 1), np.float32)
        gs, _, cnt = orc.backward(scr, snap, flags, tris, index, image, g, attr, sh, mode=ALL)
        assert cnt["intersection"] > 0 and cnt["overhang"] == 0
        alpha = pl1[:2] - pl2[:2]
        beta = pl1[2] - pl2[2]
        length = _line_length_in_square(alpha, beta, N)
        ref = -jump * pl1[0] / np.linalg.norm(alpha) * length
        est = gs[:3, 0].sum()
        err = abs(est - ref) / abs(ref)
        if not vertical_line:  # shifting triangle 2 instead: +(c1 - c2) a2_x / |grad f| * length
            ref2 = jump * pl2[0] / np.linalg.norm(alpha) * length
            err = max(err, abs(gs[3:, 0].sum() - ref2) / abs(ref2))
        errs.append(err)
    # the line crosses every pixel row, so per row one horizontal pair carries the whole crossing
    # displacement and the estimate is exact, not only convergent
    assert max(errs) < 1e-9


def test_p4_intersection_depth_shift_reading(orc):
    """Shifting triangle 1 along zeta by d: dL/dd = (c1 - c2) / |grad f| * length.  Eq. 12 applied to
    both pair orientations reproduces it for a line parallel to an image axis and gives twice it for an
    oblique line (each orientation alone already carries the full displacement)."""
    for vertical_line, factor in ((True, 1.0), (False, 2.0)):
        N = 128
        s, jump, pl1, pl2 = _intersection_scene(orc, N, vertical_line)
        scr, snap, flags, tris, index, tie, attr, sh, image = s
        g = np.ones((N, N, 1), np.float32)
        gs, _, _ = orc.backward(scr, snap, flags, tris, index, image, g, attr, sh, mode=ALL)
        alpha = pl1[:2] - pl2[:2]
        beta = pl1[2] - pl2[2]
        ref = jump / np.linalg.norm(alpha) * _line_length_in_square(alpha, beta, N)
        est = gs[:3, 2].sum()
        assert est == pytest.approx(factor * ref, rel=0.04)


# ---------------------------------------------------------------------------
# P5 finite differences of the exact box-filtered image
# ---------------------------------------------------------------------------

def _p5_scene(N):
    """Flat-depth triangles (one zeta each, so perspective interpolation is affine), per-vertex colours;
    triangle 2 partly occludes triangle 0; triangle 1 stands alone."""
    unit = np.array([[0.12, 0.15], [0.55, 0.2], [0.25, 0.62],      # 0 back
                     [0.62, 0.58], [0.9, 0.72], [0.7, 0.92],       # 1 alone
                     [0.4, 0.35], [0.72, 0.42], [0.46, 0.8]])      # 2 front of 0
    zeta = np.array([0.3] * 3 + [0.5] * 3 + [0.7] * 3)
    col = np.array([0.9, 0.4, 0.6, 0.2, 0.8, 0.5, 0.1, 0.3, 0.95])
    T = np.array([[0, 1, 2], [3, 5, 4], [6, 7, 8]], np.int32)
    return unit * N, zeta, col, T


def _box_L(P, zeta, col, T, N, w, bg, tris_subset=None, window=None):
    tris2d = [P[T[t]] for t in range(len(T))]

    def colour(t, x, y):
        Minv, _ = geom.lambda_gradients(tris2d[t])
        lam = Minv @ np.array([x, y, 1.0])
        return float(lam @ col[T[t]])

    order = sorted(range(len(T)), key=lambda t: -zeta[T[t][0]])
    if window is None:
        img = geom.box_filtered_flat(tris2d, colour, order, N, N, bg)
        return float((w * img).sum())
    (x0, x1, y0, y1) = window
    sub = np.zeros((y1 - y0, x1 - x0))
    shifted = [tp - np.array([x0, y0]) for tp in tris2d]

    def colour_s(t, x, y):
        return colour(t, x + x0, y + y0)

    sub = geom.box_filtered_flat(shifted, colour_s, order, y1 - y0, x1 - x0, bg)
    return float((w[y0:y1, x0:x1] * sub).sum())


@pytest.mark.slow
def test_p5_box_filtered_finite_differences(orc):
    """Relative error of the micro-edge gradient against central FDs of the exact box-filtered loss
    falls as the resolution doubles (the paper's accuracy metric, relative L2 error)."""
    bg = 0.05
    errs = []
    for N in (16, 32, 64):
        P, zeta, col, T = _p5_scene(N)
        yy, xx = np.mgrid[0:N, 0:N] + 0.5
        w = 1.0 + 0.5 * np.sin(2 * np.pi * xx / N) * np.cos(2 * np.pi * yy / N)
        scr = np.concatenate([P, zeta[:, None]], 1)
        s = flat_scene(orc, scr, T, N, N, col, bg)
        scr_s, snap, flags, tris, index, tie, attr, sh, image = s
        gs, _, _ = orc.backward(scr_s, snap, flags, tris, index, image, w[..., None].astype(np.float32),
                                attr, sh, mode=ALL)
        h = 1e-4 * N / 16
        fd = np.zeros((len(P), 2))
        for v in range(len(P)):
            ts = [t for t in range(len(T)) if v in T[t]] + [2]  # occluder affects the window too
            pts = np.concatenate([P[T[t]] for t in ts])
            x0 = max(0, int(np.floor(pts[:, 0].min())) - 1)
            x1 = min(N, int(np.ceil(pts[:, 0].max())) + 1)
            y0 = max(0, int(np.floor(pts[:, 1].min())) - 1)
            y1 = min(N, int(np.ceil(pts[:, 1].max())) + 1)
            for q in range(2):
                Pp = P.copy()
                Pm = P.copy()
                Pp[v, q] += h
                Pm[v, q] -= h
                fd[v, q] = (_box_L(Pp, zeta, col, T, N, w, bg, window=(x0, x1, y0, y1)) -
                            _box_L(Pm, zeta, col, T, N, w, bg, window=(x0, x1, y0, y1))) / (2 * h)
        errs.append(np.linalg.norm(gs[:, :2] - fd) / np.linalg.norm(fd))
    # measured: 38 %, 17.5 %, 9.5 % (and 4.3 % at N = 128): first-order convergence
    assert errs[-1] < 0.12
    assert all(e2 < 0.7 * e1 for e1, e2 in zip(errs, errs[1:]))


# ---------------------------------------------------------------------------
# P6 interior term against frozen-visibility finite differences
# ---------------------------------------------------------------------------

def _p6_case(orc, sc):
    r = orc.render_view(sc.verts, sc.tris, sc.cams[0], sc.H, sc.W, sc.attr, sc.shading, sc.tex)
    g = np.random.default_rng(7).standard_normal(r.image.shape).astype(np.float32)
    gs, _, _ = orc.backward(r.scr, r.snap, r.flags, sc.tris, r.index, r.image, g, sc.attr, sc.shading, sc.tex,
                            mode=INTERIOR)
    rng = np.random.default_rng(8)
    visible = np.unique(sc.tris[np.unique(r.index[r.index >= 0])])
    for v in rng.choice(visible, 12, replace=False):
        for q in range(3):
            h = 1e-6 if q < 2 else 1e-6 * r.scr[v, 2]
            sp = r.scr.copy()
            sm = r.scr.copy()
            sp[v, q] += h
            sm[v, q] -= h
            Ip = orc.shade(sp, sc.tris, r.index, sc.attr, sc.shading, sc.tex)
            Im = orc.shade(sm, sc.tris, r.index, sc.attr, sc.shading, sc.tex)
            fd = float((g * (Ip - Im)).sum()) / (2 * h)
            assert gs[v, q] == pytest.approx(fd, rel=2e-5, abs=1e-6 * (1 + abs(fd)))


def test_p6_interior_interpolated_colours(orc):
    _p6_case(orc, scenes.tiny_icosphere(H=64, W=72))


def test_p6_interior_normals_mask_depth(orc):
    _p6_case(orc, scenes.two_spheres(H=64, W=64, subdiv=2))


def test_p6_interior_texture(orc):
    sc = scenes.head_single_view(H=64, W=64, n=8, tex_size=32)
    _p6_case(orc, sc)


# ---------------------------------------------------------------------------
# P7 special cases with no edge term
# ---------------------------------------------------------------------------

def test_p7_full_screen_triangle_and_background(orc):
    N = 32
    s = flat_scene(orc, [[-40, -40, 0.5], [200, -40, 0.5], [-40, 200, 0.5]], [[0, 1, 2]], N, N, [0.7] * 3, 0.1)
    scr, snap, flags, tris, index, tie, attr, sh, image = s
    assert np.all(index == 0)
    g = np.random.default_rng(3).standard_normal((N, N, 1)).astype(np.float32)
    gs, _, cnt = orc.backward(scr, snap, flags, tris, index, image, g, attr, sh, mode=EDGE | INTERSECT)
    assert cnt["differing"] == 0 and np.all(gs == 0)
    # all background
    s = flat_scene(orc, [[-40, -40, 0.5], [-30, -40, 0.5], [-40, -30, 0.5]], [[0, 1, 2]], N, N, [0.7] * 3, 0.1)
    scr, snap, flags, tris, index, tie, attr, sh, image = s
    assert np.all(index == -1)
    gs, _, cnt = orc.backward(scr, snap, flags, tris, index, image, g, attr, sh, mode=ALL)
    assert cnt["differing"] == 0 and np.all(gs == 0)


def test_p7_coplanar_shared_edge_is_adjacent(orc):
    """Two coplanar triangles sharing an edge, same colour: every differing pair inside is adjacent."""
    N = 40
    scr = [[5.2, 5.1, 0.5], [34.7, 6.3, 0.5], [6.1, 33.9, 0.5], [35.3, 34.6, 0.5]]
    s = flat_scene(orc, scr, [[0, 1, 2], [1, 3, 2]], N, N, [0.6] * 4, 0.2)
    scr, snap, flags, tris, index, tie, attr, sh, image = s
    g = np.random.default_rng(4).standard_normal((N, N, 1)).astype(np.float32)
    gs_all, _, cnt = orc.backward(scr, snap, flags, tris, index, image, g, attr, sh, mode=EDGE | INTERSECT)
    assert cnt["adjacent"] > 20 and cnt["intersection"] == 0
    # only silhouette pairs (against background) scatter; the shared diagonal contributes nothing:
    # compare against the same square drawn as one quad-sized pair of triangles with a different split
    s2 = flat_scene(orc, [[5.2, 5.1, 0.5], [34.7, 6.3, 0.5], [6.1, 33.9, 0.5], [35.3, 34.6, 0.5]],
                    [[0, 1, 3], [0, 3, 2]], N, N, [0.6] * 4, 0.2)
    np.testing.assert_array_equal(s2[4] >= 0, index >= 0)


# ---------------------------------------------------------------------------
# Back-face image (Supp. B): a binary channel differentiable only through its edges
# ---------------------------------------------------------------------------

def _world_back_facing(sc):
    """Independent facing test in world space: the normal (v1 - v0) x (v2 - v0) points away from the camera."""
    cam = sc.cams[0]
    R = np.asarray(cam["R"], np.float64).reshape(3, 3)
    t = np.asarray(cam["t"], np.float64).reshape(3)
    centre = -R.T @ t
    V = sc.verts.astype(np.float64)
    F = sc.tris
    n = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    return (n * (centre - V[F[:, 0]])).sum(axis=1) < 0


def test_backface_image_matches_world_normals(orc):
    """Open sphere seen through its hole: the back-face channel is 1 exactly on the pixels whose visible triangle
    faces away from the camera in world space, 0 on the others and on the background; both kinds occur."""
    sc = scenes.open_sphere(H=128, W=128)
    r = orc.render(sc)[0]
    cov = r.index >= 0
    bf = _world_back_facing(sc)
    ch = r.image[..., sc.shading.backface_ch]
    np.testing.assert_array_equal(ch[cov], bf[r.index[cov]].astype(np.float64))
    assert np.all(ch[~cov] == 0.0)
    assert 0.1 < ch[cov].mean() < 0.95


def test_backface_closed_sphere_outside_and_inside(orc):
    """A closed outward-oriented sphere shows no back face from outside and only back faces from inside."""
    P, F = scenes.icosphere(3)
    sh = Shading(n_main=0, C=2, backface_ch=0, mask_ch=1, bg=[0, 0])
    attr = np.zeros((len(P), 1), np.float32)
    for eye, expect in (((0.3, 0.4, 3.0), 0.0), ((0.05, -0.03, 0.1), 1.0)):
        cam = scenes.look_at_camera(eye, 64, 64, target=(0.3, 0.2, 1.0) if expect else (0.0, 0.0, 0.0))
        r = orc.render_view(P.astype(np.float32), F, cam, 64, 64, attr, sh)
        cov = r.index >= 0
        assert cov.mean() > 0.3
        assert np.all(r.image[..., 0][cov] == expect)


@pytest.mark.parametrize("winding", [(0, 1, 2), (0, 2, 1)])
def test_backface_loss_ramp_identity(orc, winding):
    """L = sum_p x_p B_p on the back-face channel of one triangle: the x gradients sum to #covered when the
    triangle faces away (B = 1 inside, 0 outside: the P1 identity with c - bg = 1) and vanish when it faces
    the camera (B = 0 everywhere); no interior term in either case."""
    H, W = 40, 48
    pts = [[5.3, 4.1, 0.5], [41.7, 9.9, 0.5], [17.2, 35.6, 0.5]]
    scr, snap, flags = orc.snap_screen(np.asarray(pts, dtype=np.float64))
    tris = np.asarray([winding], dtype=np.int32)
    index, _, _ = orc.rasterize(scr, snap, flags, tris, H, W)
    sh = Shading(n_main=0, C=1, backface_ch=0, bg=[0.0])
    attr = np.zeros((3, 1), np.float32)
    image = orc.shade(scr, tris, index, attr, sh, snap=snap)
    X, Y = snap[:, 0].astype(np.int64), snap[:, 1].astype(np.int64)
    a, b, c = winding
    area = (X[b] - X[a]) * (Y[c] - Y[a]) - (Y[b] - Y[a]) * (X[c] - X[a])
    facing_away = area > 0  # y down: positive screen area = clockwise on the page
    yy, xx = np.mgrid[0:H, 0:W] + 0.5
    g = xx[..., None].astype(np.float32)
    gs, _, _ = orc.backward(scr, snap, flags, tris, index, image, g, attr, sh, mode=ALL)
    ncov = int((index >= 0).sum())
    assert ncov > 100
    if facing_away:
        assert np.all(image[..., 0][index >= 0] == 1.0)
        assert gs[:, 0].sum() == pytest.approx(ncov, rel=1e-12)
    else:
        assert np.all(image == 0.0)
        assert np.all(gs == 0.0)
    gi, _, _ = orc.backward(scr, snap, flags, tris, index, image, g, attr, sh, mode=INTERIOR)
    assert np.all(gi == 0.0)


# ---------------------------------------------------------------------------
# Exact-crossing gather weights (an option): same identities, faster convergence
# ---------------------------------------------------------------------------

EXACT_CROSSING = 8


@pytest.mark.parametrize("axis", [0, 1])
def test_exact_crossing_ramp_identity(orc, axis):
    """The crossing weights of each pair sum to 1, so the P1 identity stays exact."""
    H, W = 40, 48
    c, bg = 0.75, 0.25
    s = flat_scene(orc, [[5.3, 4.1, 0.5], [41.7, 9.9, 0.5], [17.2, 35.6, 0.5]], [[0, 1, 2]], H, W, [c] * 3, bg)
    scr, snap, flags, tris, index, tie, attr, sh, image = s
    yy, xx = np.mgrid[0:H, 0:W] + 0.5
    g = (xx if axis == 0 else yy)[..., None].astype(np.float32)
    gs, _, _ = orc.backward(scr, snap, flags, tris, index, image, g, attr, sh, mode=ALL | EXACT_CROSSING)
    ncov = int((index >= 0).sum())
    assert gs[:, axis].sum() == pytest.approx((c - bg) * ncov, rel=1e-12, abs=1e-9)
    assert abs(gs[:, 1 - axis].sum()) < 1e-9 * ncov
    assert np.abs(gs[:, 2]).max() < 1e-9  # overhang: no zeta component; flat colour: no interior term


def test_exact_crossing_closed_form_converges_fast(orc):
    """With exact-crossing weights the boundary gradient of P2 is within 1 % of the closed form already at
    16 px and at least 10x closer than the pixel-centre weights at every resolution."""
    c, bg = 0.75, 0.25
    unit = np.array([[0.113, 0.097], [0.871, 0.233], [0.352, 0.904]])
    for N in [16, 32, 64, 128]:
        P2 = unit * N
        scr = np.concatenate([P2, np.full((3, 1), 0.5)], axis=1)
        s = flat_scene(orc, scr, [[0, 2, 1]], N, N, [c] * 3, bg)
        scr, snap, flags, tris, index, tie, attr, sh, image = s
        g = np.ones((N, N, 1), np.float32)
        ref = (c - bg) * _area_gradient(P2)
        err = {}
        for mode in (ALL, ALL | EXACT_CROSSING):
            gs, _, _ = orc.backward(scr, snap, flags, tris, index, image, g, attr, sh, mode=mode)
            err[mode] = np.linalg.norm(gs[:, :2] - ref) / np.linalg.norm(ref)
        assert err[ALL | EXACT_CROSSING] < 0.01
        assert err[ALL | EXACT_CROSSING] < err[ALL] / 10


def _exit_point(P2, F, O):
    """Brute force: the point where the segment F -> O leaves triangle P2 (continuous geometry), by bisection
    on an FP64 point-in-triangle test."""
    def cross2(a, b):
        return a[0] * b[1] - a[1] * b[0]

    def inside(q):
        s = [cross2(P2[(i + 1) % 3] - P2[i], q - P2[i]) for i in range(3)]
        return all(v >= 0 for v in s) or all(v <= 0 for v in s)
    lo, hi = 0.0, 1.0
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if inside(F + mid * (O - F)):
            lo = mid
        else:
            hi = mid
    return F + lo * (O - F)


def test_exact_crossing_weights_equal_brute_force_derivatives(orc):
    """For every overhang pair of random triangles, the exact-crossing weights equal the derivatives of the
    brute-force exit point's pair-axis coordinate with respect to each vertex's pair-axis coordinate (central
    differences of a bisection), away from vertices and from points the snapping could move."""
    rng = np.random.default_rng(31)
    checked = 0
    for trial in range(25):
        P2 = rng.uniform(2.0, 30.0, (3, 2))
        scr, snap, flags = orc.snap_screen(np.concatenate([P2, np.full((3, 1), 0.5)], axis=1))
        tri = np.array([0, 1, 2], np.int32)
        P2 = scr[:, :2]
        for y in range(32):
            for x in range(32):
                if not orc.covers_pixel(snap, flags, tri[None], 0, x, y):
                    continue
                for axis, (dx, dy) in ((0, (1, 0)), (0, (-1, 0)), (1, (0, 1)), (1, (0, -1))):
                    ox, oy = x + dx, y + dy
                    if orc.covers_pixel(snap, flags, tri[None], 0, ox, oy):
                        continue
                    F = np.array([x + 0.5, y + 0.5])
                    O = np.array([ox + 0.5, oy + 0.5])
                    c = _exit_point(P2, F, O)
                    if np.min(np.linalg.norm(P2 - c, axis=1)) < 1e-2:
                        continue  # at a corner: the exit edge is not unique
                    if np.linalg.norm(c - F) < 1e-3 or np.linalg.norm(c - O) < 1e-3:
                        continue  # a centre on the outline: snapping decides
                    res = orc.crossing_weights(scr, snap, tri, (x, y), (ox, oy), axis)
                    assert res is not None
                    w = np.zeros(3)
                    w[res[0]] = res[1]
                    h = 1e-6
                    for k in range(3):
                        Pp, Pm = P2.copy(), P2.copy()
                        Pp[k, axis] += h
                        Pm[k, axis] -= h
                        fd = (_exit_point(Pp, F, O)[axis] - _exit_point(Pm, F, O)[axis]) / (2 * h)
                        assert fd == pytest.approx(w[k], abs=1e-5), (trial, x, y, axis, k, fd, w)
                    checked += 1
    assert checked > 200


# ---------------------------------------------------------------------------
# pixel values (barycentrics module): screen barycentrics, perspective-correct barycentrics, depth
# ---------------------------------------------------------------------------

def test_pixel_values_match_direct_solves(orc):
    """Each covered pixel's screen barycentrics solve [x; y; 1] lam = [px; py; 1]; its perspective-correct
    weights b are the affine weights of the camera-space point on the pixel ray (a direct 3x3 solve, see
    ``geom.perspective_weights``); its depth is that point's Z, and also 1 / zeta of the plane through the
    vertices in (x_s, y_s, zeta) (zeta = 1/Z is affine on screen).  Background pixels hold zeros."""
    rng = np.random.default_rng(41)
    H, W = 20, 26
    nt = 10
    V2 = rng.uniform(-6, 32, (3 * nt, 2))
    zeta = rng.uniform(0.15, 0.9, 3 * nt)  # strongly varying depth across each triangle
    scr = np.concatenate([V2, zeta[:, None]], axis=1)
    T = np.arange(3 * nt, dtype=np.int32).reshape(nt, 3)
    scr, snap, flags = orc.snap_screen(scr)
    index, _, _ = orc.rasterize(scr, snap, flags, T, H, W)
    lam, bary, depth = orc.pixel_values(scr, T, index)
    checked = 0
    for y in range(H):
        for x in range(W):
            t = index[y, x]
            if t < 0:
                assert np.all(lam[y, x] == 0) and np.all(bary[y, x] == 0) and depth[y, x] == 0
                continue
            P3 = scr[T[t]]
            px, py = x + 0.5, y + 0.5
            M = np.array([P3[:, 0], P3[:, 1], np.ones(3)])
            lam_ref = np.linalg.solve(M, np.array([px, py, 1.0]))
            b_ref, Z_ref = geom.perspective_weights(P3, px, py)
            plane = np.linalg.solve(np.array([P3[:, 0], P3[:, 1], np.ones(3)]).T, P3[:, 2])
            Z_plane = 1.0 / (plane @ np.array([px, py, 1.0]))
            np.testing.assert_allclose(lam[y, x], lam_ref, rtol=1e-9, atol=1e-11)
            np.testing.assert_allclose(bary[y, x], b_ref, rtol=1e-9, atol=1e-11)
            assert depth[y, x] == pytest.approx(Z_ref, rel=1e-11)
            assert depth[y, x] == pytest.approx(Z_plane, rel=1e-11)
            checked += 1
    assert checked > 150


# ---------------------------------------------------------------------------
# texel-cell ambiguity flags (test helper): brute-force FP32 evaluations of the texel coordinate
# ---------------------------------------------------------------------------

def _fp32_texel_coords(b, uk, N, rel_ulps, rng, draws):
    """Texel coordinate x = u N - 1/2 of u = sum_k b_k u_k as an FP32 evaluation forms it: the base
    x_0 = u_0 N - 1/2 (exact for N a power of two), the offset sum_{k=1,2} b_k (x_k - x_0) in FP32 with
    b_k carrying a relative error of up to ``rel_ulps`` ulps, added to the fraction of x_0 (the integer part
    split off exactly).  Returns the cells floor(x) of ``draws`` evaluations with random errors and of the
    four extreme sign patterns, [npix, draws + 4]."""
    f32 = np.float32
    ulp = f32(2.0 ** -24)
    x = (uk.astype(f32) * f32(N) - f32(0.5)).astype(f32)  # [npix, 3], exact
    xb = x[:, 0]
    fl = np.floor(xb)
    base = (xb - fl).astype(f32)
    pats = [rng.uniform(-1, 1, (len(b), 2)) for _ in range(draws)]
    pats += [np.tile(np.array(s, float), (len(b), 1)) for s in ((1, 1), (1, -1), (-1, 1), (-1, -1))]
    cells = []
    for p in pats:
        b1 = (b[:, 1] * (1.0 + rel_ulps * float(ulp) * p[:, 0])).astype(f32)
        b2 = (b[:, 2] * (1.0 + rel_ulps * float(ulp) * p[:, 1])).astype(f32)
        d = (b1 * (x[:, 1] - xb).astype(f32)).astype(f32) + (b2 * (x[:, 2] - xb).astype(f32)).astype(f32)
        f = (base + d.astype(f32)).astype(f32)
        cells.append(fl + np.floor(f.astype(np.float64)))
    return np.stack(cells, axis=1)


@pytest.mark.parametrize("axis", [0, 1])
def test_texel_ambiguity_flags_every_pixel_an_fp32_evaluation_can_move(orc, axis):
    """Two large triangles at constant depth (so b = lambda, affine on screen) carry uv such that the texel
    coordinate along ``axis`` is the pixel's own coordinate (minus a shift, so that on the v axis some rows
    sit on the clamp edges 0 and n - 1) plus delta, a tiny offset that grows along the other screen axis:
    many pixels lie close to a texel-cell boundary.  Each pixel whose cell (on v: the clamp state) changes
    under some FP32 evaluation of the texel coordinate (barycentric errors up to 16 ulps, FP32 operations)
    must be flagged; pixels whose offset is far beyond the flag's bound must not be."""
    H, W, N = 48, 44, 32
    shift = 0.0 if axis == 0 else 10.0
    big = 4.0 * max(H, W)
    scr = np.array([[0.0, 0.0, 0.5], [big, 0.0, 0.5], [0.0, big, 0.5], [big, big, 0.5]])
    T = np.array([[0, 1, 2], [1, 3, 2]], np.int32)
    scr, snap, flags = orc.snap_screen(scr)
    index, _, _ = orc.rasterize(scr, snap, flags, T, H, W)
    assert np.all(index >= 0)
    other = 1 - axis
    n_other = W if other == 0 else H
    alpha = 1e-5  # delta per pixel along the other axis; zero in the middle
    # texel coordinate along `axis`: P_axis - 1/2 - shift + alpha (P_other - n_other / 2)  (u = (coord + 1/2) / N)
    a = np.zeros((4, 2), np.float32)
    for v in range(4):
        coord = scr[v, axis] - 0.5 - shift + alpha * (scr[v, other] - n_other / 2)
        a[v, axis] = np.float32((coord + 0.5) / N)
        a[v, other] = np.float32((N // 2 + 0.25) / N)
    sh = Shading(n_main=3, C=3, uv_offset=0, bg=[0, 0, 0])
    tex = np.zeros((N, N, 4), np.float32)
    flagged = orc.texel_ambiguity(scr, T, index, a, sh, tex)
    ys, xs = np.mgrid[0:H, 0:W]
    b = np.zeros((H * W, 3))
    uk = np.zeros((H * W, 3))
    for i, (y, x) in enumerate(zip(ys.ravel(), xs.ravel())):
        t = index[y, x]
        M = np.array([scr[T[t], 0], scr[T[t], 1], np.ones(3)])
        b[i] = np.linalg.solve(M, np.array([x + 0.5, y + 0.5, 1.0]))
        uk[i] = a[T[t], axis]
    cells = _fp32_texel_coords(b, uk, N, 16.0, np.random.default_rng(7), 16)
    exact_x = (b * uk.astype(np.float64)).sum(axis=1) * N - 0.5
    exact = np.floor(exact_x)
    if axis == 1:  # v clamps: only the clamp state and the interior cell matter
        cells = np.clip(cells, -1, N - 1)
        exact = np.clip(exact, -1, N - 1)
    must = (cells != exact[:, None]).any(axis=1).reshape(H, W)
    assert must.sum() > 30, "the offsets should put many pixels within FP32 reach of a boundary"
    if axis == 1:
        near_low = np.abs(exact_x) < 2e-5
        assert (must.ravel() & near_low).any(), "some pixel must sit on the lower clamp edge"
    missed = must & ~flagged
    assert missed.sum() == 0, f"{int(missed.sum())} pixels can change cell but are not flagged"
    delta = np.abs(exact_x - np.rint(exact_x)).reshape(H, W)
    far = delta > 1.5e-4
    assert far.sum() > 100 and not flagged[far].any(), "pixels far from every boundary are flagged"


def test_texel_ambiguity_share_on_head_scale_view_is_small(orc):
    """On a textured head-scale view the flags touch a small share of the covered pixels (they exclude
    triangles from the gradient comparison, so their share bounds what the parity tests leave out)."""
    sc = scenes.head_single_view(H=256, W=256, n=64, tex_size=512)
    ov = orc.render(sc)[0]
    cov = ov.index >= 0
    share = ov.texamb[cov].mean()
    assert cov.sum() > 20000
    assert share < 2e-3, share


# ---------------------------------------------------------------------------
# world-space conditioning sums (test helper of the parity bound)
# ---------------------------------------------------------------------------

def test_world_condition_matches_finite_difference_jacobian(orc):
    """oracle.world_condition pushes per-view magnitude sums through |R^T J^T|; with J taken by finite
    differences of an independent homogeneous projection, the same sums agree, and they bound the world
    gradient of any per-view gradient whose magnitudes they are."""
    sc = scenes.head_multiview(n_views=3, H=64, W=48, n=8)
    views = [0, 1, 2]
    ovs = orc.render(sc, views)
    rng = np.random.default_rng(5)
    S_views = [np.abs(rng.standard_normal((len(sc.verts), 3))) for _ in views]
    Sw = orc.world_condition(sc, views, ovs, S_views)
    ref = np.zeros_like(Sw)
    gw = np.zeros_like(Sw)
    for k, v in enumerate(views):
        J = geom.projection_jacobian_fd(sc.verts, sc.cams[v])  # d(screen)/d(world)
        ref += np.einsum("vkj,vk->vj", np.abs(J), S_views[k])
        g = S_views[k] * rng.choice([-1.0, 1.0], S_views[k].shape)
        gw += orc.project_backward(sc.verts, sc.cams[v], g)
    np.testing.assert_allclose(Sw, ref, rtol=1e-6, atol=1e-9)
    assert np.all(np.abs(gw) <= Sw * (1 + 1e-9) + 1e-12)


# ---------------------------------------------------------------------------
# banded evaluation (test infrastructure for the long oracle-driven loops)
# ---------------------------------------------------------------------------

def test_banded_shading_and_backward_equal_the_whole_view(orc):
    """Shading and the backward in bands of rows on several threads give the whole-view results: the image bit
    for bit, the gradients up to the order of the FP64 sums, the pair counts exactly."""
    sc = scenes.two_spheres(H=96, W=80, subdiv=3)
    r = orc.render_view(sc.verts, sc.tris, sc.cams[0], sc.H, sc.W, sc.attr, sc.shading)
    r5 = orc.render_view(sc.verts, sc.tris, sc.cams[0], sc.H, sc.W, sc.attr, sc.shading, threads=5)
    np.testing.assert_array_equal(r.image, r5.image)
    g = sc.upstream()[0]
    a = orc.backward(r.scr, r.snap, r.flags, sc.tris, r.index, r.image, g, sc.attr, sc.shading, want_attr=True,
                     want_abs=True)
    b = orc.backward(r.scr, r.snap, r.flags, sc.tris, r.index, r.image, g, sc.attr, sc.shading, want_attr=True,
                     want_abs=True, threads=7)
    np.testing.assert_allclose(b[0], a[0], rtol=1e-12, atol=1e-12 * np.abs(a[0]).max())
    np.testing.assert_allclose(b[1], a[1], rtol=1e-12, atol=1e-12 * np.abs(a[1]).max())
    np.testing.assert_allclose(b[3], a[3], rtol=1e-12)
    assert {k: v for k, v in a[2].items() if k != "grad_attr_abs"} == \
        {k: v for k, v in b[2].items() if k != "grad_attr_abs"}
    assert a[2]["intersection"] > 0


def test_oracle_loop_normals_match_independent_formula():
    """The oracle-driven loop's FP64 vertex normals equal the input generator's numpy normals."""
    import torch

    from oracle.fitloop import vertex_normals_fp64

    sc = scenes.tiny_icosphere()
    a = vertex_normals_fp64(torch.from_numpy(sc.verts).double(), torch.from_numpy(sc.tris).long()).numpy()
    b = scenes.vertex_normals(sc.verts.astype(np.float64), sc.tris)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-14)
