"""Helpers for the GPU-vs-oracle parity tests: run one scene through the CUDA
path (C-ABI via the binding) and through the FP64 oracle, then compare.

Tolerances (written here, used by every parity test):
* index image: bit-exact on every pixel the oracle does not flag as a depth
  near-tie (relative zeta gap <= 1e-6); flagged pixels are counted.
* image and depth values: |g - o| <= 1e-5 (1 + |o|).
* vertex gradients (per view, and the world-space sum), per component, FP32
  arithmetic against FP64:  |g - o| <= 1e-6 + 1e-4 |o| + 2e-6 S, where S is the
  sum of the magnitudes of all per-pixel contributions to that component
  (computed by the oracle; for the edge term of Eq. 11 the image difference
  I_A - I_B enters as |I_A| + |I_B|, its conditioning when the image itself is
  FP32).  A component is a sum of many signed terms; when they cancel to far
  below S no FP32 evaluation of the terms can reach 1e-4 of the result, so the
  bound also admits ~34 FP32 ulps of S.
* pixels whose result is not unique are excluded with the vertices they touch:
  depth near-ties whose index differs, and pixels whose texel coordinate lies
  within the FP32 error bound of a texel-cell boundary (the bilinear derivative
  is discontinuous there; either one-sided value is correct).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

IMG_TOL = 1e-5
GRAD_ABS, GRAD_REL, GRAD_COND = 1e-6, 1e-4, 2e-6


@dataclass
class GpuResult:
    index: np.ndarray
    depth: np.ndarray
    bary: np.ndarray
    image: np.ndarray
    vpix: np.ndarray
    grad_vpix: np.ndarray
    grad_verts: np.ndarray
    grad_attr: np.ndarray | None


def gpu_run(scene, grad_images: np.ndarray, terms: int = 7, tile: int = 16, want_attr: bool = False,
            store_bary: bool = True, cover_hint: bool = True) -> GpuResult:
    import torch

    from paper_2405_02508_gb300 import binding as B
    from paper_2405_02508_gb300.render import Renderer

    dev = "cuda"
    verts = torch.from_numpy(np.ascontiguousarray(scene.verts)).to(dev)
    cams = B.cameras_tensor(scene.cams)
    attr = torch.from_numpy(np.ascontiguousarray(scene.attr)).to(dev)
    tex = torch.from_numpy(scene.tex).to(dev) if scene.tex is not None else None
    n, H, W = scene.n_views, scene.H, scene.W
    r = Renderer(torch.from_numpy(scene.tris), len(scene.verts), n, H, W, scene.shading, scene.attr.shape[1],
                 None if tex is None else tex.shape, tile=tile, cover_hint=cover_hint)
    depth = torch.empty((n, H, W), dtype=torch.float32, device=dev)
    bary = torch.empty((n, H, W, 2), dtype=torch.float32, device=dev) if store_bary else None
    r.forward(verts, cams, attr, tex, depth=depth, bary=bary)
    g = torch.from_numpy(np.ascontiguousarray(grad_images, dtype=np.float32)).to(dev)
    ga = torch.zeros_like(attr) if want_attr else None
    r.backward(g, cams, attr, tex, terms=terms, grad_attr=ga)
    r.check_status()
    torch.cuda.synchronize()
    return GpuResult(r.index.cpu().numpy(), depth.cpu().numpy(), None if bary is None else bary.cpu().numpy(),
                     r.image.cpu().numpy(), r.vpix.cpu().numpy(), r.grad_vpix.cpu().numpy(),
                     r.grad_verts.cpu().numpy(), None if ga is None else ga.cpu().numpy())


def excluded_vertices(tris, idx_a, idx_b, ambiguous=None):
    """Vertices whose gradients may legitimately differ: triangles at pixels where the two index images
    differ (flagged near-ties) and at their 4-neighbours, and triangles at texel-ambiguous pixels."""
    diff = idx_a != idx_b
    extra = np.zeros(0, np.int64)
    if ambiguous is not None and ambiguous.any():
        ts = np.unique(idx_b[ambiguous & (idx_b >= 0)])
        extra = np.unique(tris[ts].reshape(-1))
    if not diff.any():
        return extra
    m = diff.copy()
    m[1:, :] |= diff[:-1, :]
    m[:-1, :] |= diff[1:, :]
    m[:, 1:] |= diff[:, :-1]
    m[:, :-1] |= diff[:, 1:]
    ts = np.unique(np.concatenate([idx_a[m], idx_b[m]]))
    ts = ts[ts >= 0]
    return np.unique(np.concatenate([tris[ts].reshape(-1), extra]))


def grad_violations(g: np.ndarray, o: np.ndarray, S=None, exclude=None):
    """Returns (number of violating components, worst |g-o| / bound)."""
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    S = np.zeros_like(o) if S is None else np.asarray(S, np.float64)
    if exclude is not None and len(exclude):
        keep = np.ones(len(o), bool)
        keep[exclude] = False
        g, o, S = g[keep], o[keep], S[keep]
    ratio = np.abs(g - o) / (GRAD_ABS + GRAD_REL * np.abs(o) + GRAD_COND * S)
    return int((ratio > 1.0).sum()), float(ratio.max() if ratio.size else 0.0)


def compare_view(gpu: GpuResult, view: int, ov, orc_grad_scr, tris, check_grad=True, S=None):
    """Compare one view; returns a dict of statistics and asserts the parity bar."""
    gi = gpu.index[view]
    oi = ov.index
    tie = ov.tie
    mism = (gi != oi) & ~tie
    assert mism.sum() == 0, f"view {view}: {int(mism.sum())} index mismatches outside near-ties"
    same = gi == oi
    cov = same & (oi >= 0)
    dd = np.abs(gpu.depth[view][cov] - ov.depth[cov]) / (1 + np.abs(ov.depth[cov]))
    assert dd.size == 0 or dd.max() <= IMG_TOL, f"view {view}: depth error {dd.max()}"
    di = np.abs(gpu.image[view][same] - ov.image[same]) / (1 + np.abs(ov.image[same]))
    assert di.size == 0 or di.max() <= IMG_TOL, f"view {view}: image error {di.max()}"
    if gpu.bary is not None:
        db = np.abs(gpu.bary[view][cov] - ov.bary[cov][:, 1:]).max() if cov.any() else 0.0
        assert db <= IMG_TOL, f"view {view}: bary error {db}"
    stats = {"ties": int(tie.sum()), "tie_mismatch": int((gi != oi).sum()), "covered": int((oi >= 0).sum())}
    if check_grad:
        ex = excluded_vertices(tris, gi, oi, getattr(ov, "texamb", None))
        nbad, worst = grad_violations(gpu.grad_vpix[view], orc_grad_scr, S, ex)
        stats.update(grad_bad=nbad, grad_worst=worst, excluded=len(ex))
        assert nbad == 0, f"view {view}: {nbad} gradient components outside tolerance (worst ratio {worst:.3g})"
    return stats


def world_condition(scene, views, ovs, S_views):
    import oracle

    return oracle.world_condition(scene, views, ovs, S_views)
