"""Pins of the oracle's forward gradients (per-pixel image derivative along one scene parameter, Sec. 5):
exactly the transpose of the pinned backward (dot-product test), a closed form for a translated flat
triangle, and the projection tangent against finite differences and its own transpose."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2405_02508_gb300 import scenes
from paper_2405_02508_gb300.scenes import Shading

EDGE, INTERIOR, INTERSECT = 1, 2, 4
ALL = EDGE | INTERIOR | INTERSECT


def _small(name):
    if name == "two_spheres":
        return scenes.two_spheres(H=96, W=96, subdiv=3)
    if name == "textured_head":
        return scenes.head_single_view(H=96, W=96, n=16, tex_size=32)
    if name == "open_sphere":
        return scenes.open_sphere(H=96, W=96, subdiv=3)
    return scenes.tiny_icosphere(H=64, W=64)


@pytest.mark.parametrize("name", ["tiny", "two_spheres", "textured_head", "open_sphere"])
@pytest.mark.parametrize("mode", [ALL, EDGE | INTERIOR, EDGE | INTERSECT, INTERIOR])
def test_forward_grad_is_transpose_of_backward(orc, name, mode):
    """sum_p g_p . JVP(t)_p = sum_v backward(g)_v . t_v for random g and t (FP64, to rounding)."""
    sc = _small(name)
    r = orc.render(sc)[0]
    rng = np.random.default_rng(7)
    g = rng.standard_normal((sc.H, sc.W, sc.shading.C)).astype(np.float32)
    t = rng.standard_normal((len(sc.verts), 3))
    t[:, 2] *= 1e-2  # zeta is ~1/Z: keep the tangent on the same relative scale
    tex = getattr(sc, "tex", None)
    gs, _, _ = orc.backward(r.scr, r.snap, r.flags, sc.tris, r.index, r.image, g, sc.attr, sc.shading, tex,
                            mode=mode)
    jv, mag = orc.forward_grad(r.scr, r.snap, r.flags, sc.tris, r.index, r.image, t, sc.attr, sc.shading, tex,
                               mode=mode, want_abs=True)
    lhs = float((g.astype(np.float64) * jv).sum())
    rhs = float((gs * t).sum())
    scale = float((np.abs(g) * mag).sum())
    assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs, scale)
    assert scale > 0


def test_forward_grad_translated_flat_triangle_closed_form(orc):
    """Unit x translation of a flat triangle over the background: every horizontal pair (L, R) that straddles
    the outline gets 1/2 (I_L - I_R) at both pixels, vertical pairs and the interior nothing."""
    H, W = 40, 48
    c, bg = 0.75, 0.25
    scr, snap, flags = orc.snap_screen(np.array([[5.3, 4.1, 0.5], [41.7, 9.9, 0.5], [17.2, 35.6, 0.5]]))
    tris = np.array([[0, 1, 2]], np.int32)
    index, _, _ = orc.rasterize(scr, snap, flags, tris, H, W)
    sh = Shading(n_main=1, C=1, bg=[bg])
    attr = np.full((3, 1), c, np.float32)
    image = orc.shade(scr, tris, index, attr, sh)
    t = np.tile([[1.0, 0.0, 0.0]], (3, 1))
    jv = orc.forward_grad(scr, snap, flags, tris, index, image, t, attr, sh)[..., 0]
    expect = np.zeros((H, W))
    for y in range(H):
        for x in range(W - 1):
            if index[y, x] != index[y, x + 1]:
                h = 0.5 * (image[y, x, 0] - image[y, x + 1, 0])
                expect[y, x] += h
                expect[y, x + 1] += h
    np.testing.assert_allclose(jv, expect, rtol=0, atol=1e-12)
    assert np.count_nonzero(expect) > 40


def test_project_jvp_matches_finite_differences_and_transpose(orc):
    rng = np.random.default_rng(5)
    verts = rng.uniform(-1, 1, (200, 3)).astype(np.float32)
    tw = rng.standard_normal((200, 3))
    for cam in scenes.cameras_on_sphere(3, 3.0, 120, 90, seed=9):
        ts = orc.project_jvp(verts, cam, tw)
        # fourth-order central differences; the projection takes FP32 positions, so the step stays large
        h = 1e-2
        f = {k: orc.project(verts.astype(np.float64) + k * h * tw, cam)[0] for k in (-2, -1, 1, 2)}
        fd = (8.0 * (f[1] - f[-1]) - (f[2] - f[-2])) / (12.0 * h)
        np.testing.assert_allclose(ts, fd, rtol=0, atol=2e-5 * np.abs(fd).max())
        g = rng.standard_normal((200, 3))
        gw = orc.project_backward(verts, cam, g)
        assert float((g * ts).sum()) == pytest.approx(float((gw * tw).sum()), rel=1e-12)


@pytest.mark.parametrize("name", ["tiny", "two_spheres", "open_sphere"])
def test_forward_grad_exact_crossing_is_transpose(orc, name):
    """The exact-crossing option keeps forward and backward transposes of each other."""
    sc = _small(name)
    r = orc.render(sc)[0]
    rng = np.random.default_rng(8)
    g = rng.standard_normal((sc.H, sc.W, sc.shading.C)).astype(np.float32)
    t = rng.standard_normal((len(sc.verts), 3))
    mode = ALL | 8
    gs, _, _ = orc.backward(r.scr, r.snap, r.flags, sc.tris, r.index, r.image, g, sc.attr, sc.shading, mode=mode)
    jv, mag = orc.forward_grad(r.scr, r.snap, r.flags, sc.tris, r.index, r.image, t, sc.attr, sc.shading,
                               mode=mode, want_abs=True)
    lhs, rhs = float((g.astype(np.float64) * jv).sum()), float((gs * t).sum())
    assert abs(lhs - rhs) <= 1e-12 * float((np.abs(g) * mag).sum())
    gs0, _, _ = orc.backward(r.scr, r.snap, r.flags, sc.tris, r.index, r.image, g, sc.attr, sc.shading, mode=ALL)
    assert np.abs(gs - gs0).max() > 0  # the option changes the result
