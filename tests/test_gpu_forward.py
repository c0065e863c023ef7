"""Forward gradients on the device (mer_project_jvp + mer_forward_grad) against the FP64 oracle, pixel by
pixel, and against the device backward by the dot-product test."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2405_02508_gb300 import scenes

pytestmark = pytest.mark.gpu

FWD_ABS, FWD_REL, FWD_COND = 1e-6, 1e-4, 2e-6


@pytest.fixture(scope="module")
def orc():
    import oracle

    oracle.build()
    return oracle


def _scene(name):
    if name == "two_spheres":
        return scenes.two_spheres(H=256, W=256, subdiv=4)
    if name == "textured_head":
        return scenes.head_single_view(H=256, W=256, n=32, tex_size=128)
    if name == "open_sphere":
        return scenes.open_sphere(H=256, W=256)
    return scenes.tiny_icosphere()


def _tangent(sc, kind):
    V = len(sc.verts)
    if kind == "translate_part":  # move one object (the second sphere, or the upper half) rigidly
        t = np.zeros((V, 3))
        sel = np.arange(V) >= V // 2 if sc.name.startswith("two_spheres") else sc.verts[:, 1] > 0
        t[sel] = [0.3, -0.2, 0.1]
        return t
    return np.random.default_rng(17).standard_normal((V, 3)) * 0.1


def _gpu(sc, tangent, terms=7):
    import torch

    from paper_2405_02508_gb300 import binding as B
    from paper_2405_02508_gb300.render import Renderer

    verts = torch.from_numpy(np.ascontiguousarray(sc.verts)).cuda()
    cams = B.cameras_tensor(sc.cams)
    attr = torch.from_numpy(np.ascontiguousarray(sc.attr)).cuda()
    tex = torch.from_numpy(sc.tex).cuda() if sc.tex is not None else None
    r = Renderer(torch.from_numpy(sc.tris), len(sc.verts), sc.n_views, sc.H, sc.W, sc.shading, sc.attr.shape[1],
                 None if tex is None else tex.shape)
    r.forward(verts, cams, attr, tex)
    out = r.forward_grad(torch.from_numpy(tangent.astype(np.float32)).cuda(), cams, attr, tex, terms)
    r.check_status()
    return r, out, cams, attr, tex


@pytest.mark.parametrize("name", ["tiny", "two_spheres", "textured_head", "open_sphere"])
@pytest.mark.parametrize("kind", ["translate_part", "random", "random_exact_crossing"])
def test_forward_grad_matches_oracle(orc, name, kind):
    sc = _scene(name)
    terms = 7 | (8 if kind.endswith("exact_crossing") else 0)
    t = _tangent(sc, kind)
    r, out, _, _, _ = _gpu(sc, t, terms)
    ov = orc.render(sc)[0]
    ts = orc.project_jvp(sc.verts, sc.cams[0], t)
    jv, mag = orc.forward_grad(ov.scr, ov.snap, ov.flags, sc.tris, ov.index, ov.image, ts, sc.attr, sc.shading,
                               sc.tex, mode=terms, want_abs=True)
    g = out[0].cpu().numpy().astype(np.float64)
    gi = r.index[0].cpu().numpy()
    # pixels whose result is not unique: depth near-ties (and their neighbours, whose pairs they enter) and
    # texel-ambiguous pixels
    bad = gi != ov.index
    bad = bad | np.roll(bad, 1, 0) | np.roll(bad, -1, 0) | np.roll(bad, 1, 1) | np.roll(bad, -1, 1)
    if ov.texamb is not None:
        bad |= ov.texamb.astype(bool)
    keep = ~bad
    tol = FWD_ABS * np.abs(jv).max() + FWD_REL * np.abs(jv) + FWD_COND * mag
    viol = (np.abs(g - jv) > tol) & keep[..., None]
    assert not viol.any(), (int(viol.sum()), float(np.abs(g - jv)[viol].max()))
    assert np.abs(jv[keep]).max() > 0 and bad.mean() < 0.01


@pytest.mark.parametrize("name", ["two_spheres", "textured_head"])
@pytest.mark.parametrize("terms", [7, 15])
def test_forward_grad_is_transpose_of_device_backward(name, terms):
    """sum_p g_p . JVP(t)_p = sum_v grad_world(g)_v . t_v with both sides from the device kernels."""
    import torch

    sc = _scene(name)
    t = _tangent(sc, "random")
    r, out, cams, attr, tex = _gpu(sc, t, terms)
    g = torch.from_numpy(sc.upstream()).cuda()
    gw = r.backward(g, cams, attr, tex, terms).double().cpu().numpy()
    lhs = float((g.double() * out.double()).sum())
    rhs = float((gw * t).sum())
    scale = float((g.double().abs() * out.double().abs()).sum())
    assert abs(lhs - rhs) <= 1e-4 * scale, (lhs, rhs, scale)
