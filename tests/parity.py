"""Helpers for the GPU-vs-oracle parity tests: run one scene through the CUDA
path (C-ABI via the binding) and through the FP64 oracle, then compare.

Tolerances (written here, used by every parity test):
* index image: bit-exact on every pixel the oracle does not flag as a depth
  near-tie (relative zeta gap <= 1e-6); flagged pixels are counted, and their
  share of the covered pixels of a configuration's compared views must stay
  below TIE_SHARE_MAX (``assert_tie_share``; a single small view holds too few
  pixels for a share on its own).
* image and depth values: |g - o| <= 1e-5 (1 + |o|).  With the deterministic
  option (FP64 shading rounded once) the image must equal the oracle's image
  rounded to FP32 except for values within one FP32 ulp (or 1e-9) of the
  oracle's FP64 value, at most IMG_ULP_SHARE_MAX of them: the vertex positions
  reach the kernels as snapped integers plus FP32 residuals (within 2^-33 px of
  the oracle's FP64 positions), so the FP64 values differ from the oracle's by
  ~1e-10 of the terms they sum, and a value that close to an FP32 rounding
  boundary (or a value that cancels to near zero) can round the other way.
* vertex gradients (per view, and the world-space sum), per component:
  - with the deterministic option (FP64 per-pixel arithmetic, exact sums) the
    stated bound |g - o| <= 1e-6 + 1e-4 |o|, nothing more;
  - on the default FP32 path |g - o| <= 1e-6 + 1e-4 |o| + 2e-6 S, where S is
    the sum of the magnitudes of all per-pixel contributions to that component
    (computed by the oracle; for the edge term of Eq. 11 the image difference
    I_A - I_B enters as |I_A| + |I_B|, its conditioning when the image itself is
    FP32).  A component is a sum of many signed terms; when they cancel to far
    below S no FP32 evaluation of the terms can reach 1e-4 of the result, so the
    bound also admits ~34 FP32 ulps of S.  Every comparison also counts the
    components that fail the stated bound without the S term (``strict_fail``)
    and the largest share of a component's bound that the S term supplies.
* pixels whose result is not unique are excluded with the vertices they touch:
  depth near-ties whose index differs, and pixels whose texel coordinate lies
  within the error bound of a texel-cell boundary (the bilinear derivative is
  discontinuous there; either one-sided value is correct), the bound being that
  of the arithmetic used (FP32 on the default path, FP64 with the
  deterministic option).  The excluded vertices' share is bounded:
  EXCLUDED_SHARE_MAX (deterministic) or EXCLUDED_SHARE_MAX_FP32 (default path)
  of the mesh's vertices per view.

Every comparison appends its statistics to ``LOG``; the session prints them as a
table at the end (and writes them as JSON to $MER_PARITY_LOG when set).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

IMG_TOL = 1e-5
GRAD_ABS, GRAD_REL, GRAD_COND = 1e-6, 1e-4, 2e-6
TIE_SHARE_MAX = 1e-4
EXCLUDED_SHARE_MAX = 1e-3
EXCLUDED_SHARE_MAX_FP32 = 5e-3
IMG_ULP_SHARE_MAX = 1e-3
DETERMINISTIC = 16

LOG: list[dict] = []


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
    """The scene through the per-view path; ``terms`` with the deterministic bit also selects FP64 shading."""
    import torch

    from paper_2405_02508_gb300 import binding as B
    from paper_2405_02508_gb300.render import Renderer

    dev = "cuda"
    det = bool(terms & DETERMINISTIC)
    verts = torch.from_numpy(np.ascontiguousarray(scene.verts)).to(dev)
    cams = B.cameras_tensor(scene.cams)
    attr = torch.from_numpy(np.ascontiguousarray(scene.attr)).to(dev)
    tex = torch.from_numpy(scene.tex).to(dev) if scene.tex is not None else None
    n, H, W = scene.n_views, scene.H, scene.W
    r = Renderer(torch.from_numpy(scene.tris), len(scene.verts), n, H, W, scene.shading, scene.attr.shape[1],
                 None if tex is None else tex.shape, tile=tile, cover_hint=cover_hint, precise=det)
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


def oracle_image(ov, deterministic: bool) -> np.ndarray:
    """The image the oracle's backward is given: its own FP64 image, or, with the deterministic option, that
    image rounded to FP32 (the image passed through the edge step is an FP32 tensor, and the deterministic
    option's FP64 shading produces exactly the rounded values)."""
    return ov.image.astype(np.float32).astype(np.float64) if deterministic else ov.image


def ambiguous(ov, deterministic: bool):
    return ov.texamb64 if deterministic else ov.texamb


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


def grad_violations(g: np.ndarray, o: np.ndarray, S=None, exclude=None, cond: float = GRAD_COND):
    """Returns (number of violating components, worst |g-o| / bound) for the bound
    GRAD_ABS + GRAD_REL |o| + cond S (cond = 0: the stated bound alone)."""
    st = grad_stats(g, o, S, exclude, cond)
    return st["bad"], st["worst"]


def grad_stats(g: np.ndarray, o: np.ndarray, S=None, exclude=None, cond: float = GRAD_COND) -> dict:
    """Violations of GRAD_ABS + GRAD_REL |o| + cond S, the worst ratio, the components failing the stated bound
    GRAD_ABS + GRAD_REL |o| (no S term), and the largest share of a component's bound the S term supplies
    among the components that need it."""
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    S = np.zeros_like(o) if S is None else np.asarray(S, np.float64)
    if exclude is not None and len(exclude):
        keep = np.ones(len(o), bool)
        keep[exclude] = False
        g, o, S = g[keep], o[keep], S[keep]
    err = np.abs(g - o)
    strict = GRAD_ABS + GRAD_REL * np.abs(o)
    bound = strict + cond * S
    ratio = err / bound
    need = err > strict
    share = (cond * S[need] / bound[need]).max() if need.any() else 0.0
    return {"bad": int((ratio > 1.0).sum()), "worst": float(ratio.max() if ratio.size else 0.0),
            "strict_fail": int(need.sum()), "cond_share_max": float(share), "components": int(o.size),
            "worst_strict": float((err / strict).max() if err.size else 0.0)}


def assert_tie_share(stats: list[dict]):
    """Flagged depth near-ties over the covered pixels of a configuration's compared views."""
    ties = sum(s["ties"] for s in stats)
    cov = sum(s["covered"] for s in stats)
    share = ties / max(cov, 1)
    assert share < TIE_SHARE_MAX, f"flagged depth ties: {ties} of {cov} covered pixels ({share:.2e})"
    return share


def image_rounding_mismatches(gim: np.ndarray, oim: np.ndarray):
    """(values not equal to the oracle's FP64 value rounded to FP32, values further than one FP32 ulp and 1e-9
    from it)."""
    o32 = oim.astype(np.float32)
    ne = gim.astype(np.float32) != o32
    d = np.abs(gim.astype(np.float64) - oim.astype(np.float64))
    far = d > np.maximum(np.abs(np.spacing(o32)).astype(np.float64), 1e-9)
    return ne, far


def compare_view(gpu: GpuResult, view: int, ov, orc_grad_scr, tris, check_grad=True, S=None,
                 deterministic: bool = False, label: str = "view") -> dict:
    """Compare one view; returns a dict of statistics (also appended to LOG) and asserts the parity bar."""
    gi = gpu.index[view]
    oi = ov.index
    tie = ov.tie
    mism = (gi != oi) & ~tie
    assert mism.sum() == 0, f"view {view}: {int(mism.sum())} index mismatches outside near-ties"
    same = gi == oi
    cov = same & (oi >= 0)
    ncov = int((oi >= 0).sum())
    if gpu.depth is not None:
        dd = np.abs(gpu.depth[view][cov] - ov.depth[cov]) / (1 + np.abs(ov.depth[cov]))
        assert dd.size == 0 or dd.max() <= IMG_TOL, f"view {view}: depth error {dd.max()}"
    gim = gpu.image[view][same]
    oim = ov.image[same]
    di = np.abs(gim - oim) / (1 + np.abs(oim))
    assert di.size == 0 or di.max() <= IMG_TOL, f"view {view}: image error {di.max()}"
    stats = {"label": label, "view": int(view), "deterministic": bool(deterministic), "covered": ncov,
             "ties": int(tie.sum()), "tie_share": float(tie.sum() / max(ncov, 1)),
             "tie_mismatch": int((gi != oi).sum())}
    if deterministic and gim.size:
        ne, far = image_rounding_mismatches(gim, oim)
        stats["image_ulp1"] = int(ne.sum())
        assert not far.any(), f"view {view}: {int(far.sum())} image values more than one FP32 ulp off"
        assert ne.mean() <= IMG_ULP_SHARE_MAX, f"view {view}: {int(ne.sum())} image values not correctly rounded"
    if gpu.bary is not None:
        db = np.abs(gpu.bary[view][cov] - ov.bary[cov][:, 1:]).max() if cov.any() else 0.0
        assert db <= IMG_TOL, f"view {view}: bary error {db}"
    if check_grad:
        amb = ambiguous(ov, deterministic)
        ex = excluded_vertices(tris, gi, oi, amb)
        nv = len(orc_grad_scr)
        st = grad_stats(gpu.grad_vpix[view], orc_grad_scr, S, ex, 0.0 if deterministic else GRAD_COND)
        stats.update(texamb=int(amb.sum()), texamb_share=float(amb.sum() / max(ncov, 1)), excluded=len(ex),
                     excluded_share=float(len(ex) / max(nv, 1)), grad_bad=st["bad"], grad_worst=st["worst"],
                     strict_fail=st["strict_fail"], cond_share_max=st["cond_share_max"],
                     worst_strict=st["worst_strict"], components=st["components"])
        LOG.append(stats)
        lim = EXCLUDED_SHARE_MAX if deterministic else EXCLUDED_SHARE_MAX_FP32
        assert stats["excluded_share"] < lim, f"view {view}: excluded vertices {stats['excluded_share']:.2e}"
        assert st["bad"] == 0, (f"view {view}: {st['bad']} gradient components outside tolerance "
                                f"(worst ratio {st['worst']:.3g})")
    else:
        LOG.append(stats)
    return stats


def world_condition(scene, views, ovs, S_views):
    import oracle

    return oracle.world_condition(scene, views, ovs, S_views)
