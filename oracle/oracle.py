"""Python wrapper of the FP64 CPU oracle (``oracle.c``).  TEST INFRASTRUCTURE.

Only the test suite, the package smoke check and the benchmark's CPU-baseline
leg use it.  It shares no code with the CUDA path: it takes the same seeded
scenes (``paper_2405_02508_gb300.scenes``) and computes, per view and in FP64,

* projection and snapping (vertex transform module, Supp. B),
* the index image with the stated fill rule and depth tie-break, plus the
  near-tie flags (rasterization module),
* barycentrics, depth and the shaded image (barycentrics / interpolation
  modules and deferred shading),
* the backward pass: micro-edge term (Eq. 11, Sec. 4.3 classification, Eq. 12
  for intersections) and the interior term Omega by forward-mode dual numbers,
* the projection backward.

Views are independent; ``render``/``backward`` run them on a thread pool (the C
calls release the GIL).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

EDGE, INTERIOR, INTERSECT, EXACT_CROSSING = 1, 2, 4, 8
VALID = 3


class OrcCamera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3), ("fx", ctypes.c_double),
                ("fy", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("znear", ctypes.c_double)]


class OrcShading(ctypes.Structure):
    _fields_ = [("n_main", ctypes.c_int), ("C", ctypes.c_int), ("uv_offset", ctypes.c_int),
                ("mask_ch", ctypes.c_int), ("depth_ch", ctypes.c_int), ("C_attr", ctypes.c_int),
                ("tex_h", ctypes.c_int), ("tex_w", ctypes.c_int), ("tex_c", ctypes.c_int),
                ("backface_ch", ctypes.c_int)]


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (no fused multiply-add, IEEE double)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = os.environ.get("ORACLE_LIB")  # a deliberately mutated build, used by the pin-sensitivity test
        if not path:
            path = build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i = ctypes.c_int
        L.orc_project.argtypes = [P, i, ctypes.POINTER(OrcCamera), P, P, P]
        L.orc_project.restype = None
        L.orc_covers_pixel.argtypes = [P, P, P, i, i, i]
        L.orc_covers_pixel.restype = i
        L.orc_rasterize.argtypes = [P, P, P, i, P, i, i, i, P, P, P]
        L.orc_rasterize.restype = i
        L.orc_pixel_values.argtypes = [P, P, P, i, i, P, P, P]
        L.orc_pixel_values.restype = i
        L.orc_shade.argtypes = [P, P, P, P, i, i, P, P, P, ctypes.POINTER(OrcShading), P]
        L.orc_shade.restype = i
        L.orc_shade_rows.argtypes = [P, P, P, P, i, i, P, P, P, ctypes.POINTER(OrcShading), P, i, i]
        L.orc_shade_rows.restype = i
        L.orc_backward.argtypes = [P, P, P, i, P, P, i, i, P, P, P, P, ctypes.POINTER(OrcShading), i, P, P, P, P, P]
        L.orc_backward_rows.argtypes = [P, P, P, i, P, P, i, i, P, P, P, P, ctypes.POINTER(OrcShading), i, P, P, P,
                                        P, P, i, i]
        L.orc_backward_rows.restype = i
        L.orc_texel_ambiguity.argtypes = [P, P, P, i, i, P, ctypes.POINTER(OrcShading), ctypes.c_double, P]
        L.orc_texel_ambiguity.restype = i
        L.orc_backward.restype = i
        L.orc_project_backward.argtypes = [P, i, ctypes.POINTER(OrcCamera), P, P]
        L.orc_project_backward.restype = None
        L.orc_forward_grad.argtypes = [P, P, P, i, P, P, i, i, P, P, P, ctypes.POINTER(OrcShading), i, P, P, P]
        L.orc_forward_grad.restype = i
        L.orc_crossing_weights.argtypes = [P, P, P, i, i, i, i, i, P, P]
        L.orc_crossing_weights.restype = i
        L.orc_project_jvp.argtypes = [P, i, ctypes.POINTER(OrcCamera), P, P]
        L.orc_project_jvp.restype = None
        _lib = L
    return _lib


def _p(a: np.ndarray | None):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def camera(cam) -> OrcCamera:
    c = OrcCamera()
    c.R[:] = [float(x) for x in np.asarray(cam["R"]).reshape(9)]
    c.t[:] = [float(x) for x in np.asarray(cam["t"]).reshape(3)]
    c.fx, c.fy, c.cx, c.cy, c.znear = (float(cam[k]) for k in ("fx", "fy", "cx", "cy", "znear"))
    return c


def shading(sh, C_attr: int, tex: np.ndarray | None) -> OrcShading:
    s = OrcShading()
    s.n_main, s.C, s.uv_offset, s.mask_ch, s.depth_ch = sh.n_main, sh.C, sh.uv_offset, sh.mask_ch, sh.depth_ch
    s.C_attr = C_attr
    s.tex_h, s.tex_w = (tex.shape[0], tex.shape[1]) if tex is not None else (0, 0)
    s.tex_c = tex.shape[2] if tex is not None else 0
    s.backface_ch = getattr(sh, "backface_ch", -1)
    return s


# ---------------------------------------------------------------------------
# per-view steps
# ---------------------------------------------------------------------------

def project(verts: np.ndarray, cam):
    """-> scr [V,3] f64 (x_s, y_s, zeta), snap [V,2] int64, flags [V] int32."""
    verts = np.ascontiguousarray(verts, dtype=np.float32)
    V = len(verts)
    scr = np.zeros((V, 3), np.float64)
    snap = np.zeros((V, 2), np.int64)
    flags = np.zeros(V, np.int32)
    c = camera(cam)
    lib().orc_project(_p(verts), V, ctypes.byref(c), _p(scr), _p(snap), _p(flags))
    return scr, snap, flags


def snap_screen(scr: np.ndarray, guard: float = 2.0 ** 29):
    """Snap given FP64 screen positions (screen-space input path): same rule as ``project``."""
    scr = np.ascontiguousarray(scr, dtype=np.float64)
    X = scr[:, :2] * 256.0
    ok = (np.abs(X) <= guard).all(axis=1) & (scr[:, 2] > 0)
    snap = np.where(ok[:, None], np.rint(np.where(ok[:, None], X, 0.0)), 0).astype(np.int64)
    flags = np.where(ok, VALID, np.where(scr[:, 2] > 0, 1, 0)).astype(np.int32)
    return scr, snap, flags


def rasterize(scr, snap, flags, tris, H: int, W: int):
    """-> index [H,W] int32, tie [H,W] bool, zeta_test of the winner [H,W] f64."""
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    index = np.empty((H, W), np.int32)
    zb = np.empty((H, W), np.float64)
    tie = np.empty((H, W), np.uint8)
    rc = lib().orc_rasterize(_p(scr), _p(snap), _p(flags), len(scr), _p(tris), len(tris), H, W,
                             _p(index), _p(zb), _p(tie))
    assert rc == 0
    return index, tie.astype(bool), zb


def covers_pixel(snap, flags, tris, t: int, x: int, y: int) -> bool:
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    return bool(lib().orc_covers_pixel(_p(snap), _p(flags), _p(tris), t, x, y))


def pixel_values(scr, tris, index):
    """-> lam [H,W,3] screen barycentrics, bary [H,W,3] perspective-correct, depth [H,W]."""
    H, W = index.shape
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    index = np.ascontiguousarray(index, dtype=np.int32)
    lam = np.empty((H, W, 3))
    bary = np.empty((H, W, 3))
    depth = np.empty((H, W))
    lib().orc_pixel_values(_p(scr), _p(tris), _p(index), H, W, _p(lam), _p(bary), _p(depth))
    return lam, bary, depth


def _bands(H: int, threads: int | None):
    n = max(1, min(threads or 1, H))
    edges = np.linspace(0, H, n + 1).astype(int)
    return [(int(a), int(b)) for a, b in zip(edges[:-1], edges[1:]) if b > a]


def shade(scr, tris, index, attr, sh, tex=None, snap=None, threads: int | None = None):
    """Shaded image [H,W,C] f64; ``snap`` (snapped coordinates) is needed for a back-face channel.  With
    ``threads`` > 1 the rows are shaded in bands on a thread pool (the same values)."""
    H, W = index.shape
    attr = np.ascontiguousarray(attr, dtype=np.float32)
    tex = None if tex is None else np.ascontiguousarray(tex, dtype=np.float32)
    bg = np.ascontiguousarray(sh.bg_array())
    s = shading(sh, attr.shape[1], tex)
    img = np.empty((H, W, sh.C))
    snap_c = None if snap is None else np.ascontiguousarray(snap, dtype=np.int64)
    tris_c = np.ascontiguousarray(tris, dtype=np.int32)
    index_c = np.ascontiguousarray(index, dtype=np.int32)

    def band(rows):
        return lib().orc_shade_rows(_p(scr), _p(snap_c), _p(tris_c), _p(index_c), H, W, _p(attr), _p(tex), _p(bg),
                                    ctypes.byref(s), _p(img), rows[0], rows[1])

    bands = _bands(H, threads)
    if len(bands) == 1:
        rcs = [band(bands[0])]
    else:
        with _pool(len(bands)) as ex:
            rcs = list(ex.map(band, bands))
    assert all(rc == 0 for rc in rcs)
    return img


def backward(scr, snap, flags, tris, index, image, grad_image, attr, sh, tex=None,
             mode: int = EDGE | INTERIOR | INTERSECT, want_attr: bool = False, want_abs: bool = False,
             threads: int | None = None):
    """-> grad_scr [V,3] f64, grad_attr [V,C_attr] or None, counts dict (+ grad_abs [V,3] if want_abs:
    the sum of the absolute values of every per-pixel contribution, the conditioning of each sum).  With
    ``threads`` > 1 bands of rows run on a thread pool, each into its own sums, added at the end (the same
    result up to the order of the FP64 additions)."""
    H, W = index.shape
    V = len(scr)
    attr = np.ascontiguousarray(attr, dtype=np.float32)
    tex = None if tex is None else np.ascontiguousarray(tex, dtype=np.float32)
    image = np.ascontiguousarray(image, dtype=np.float64)
    grad_image = np.ascontiguousarray(grad_image, dtype=np.float32)
    tris_c = np.ascontiguousarray(tris, dtype=np.int32)
    index_c = np.ascontiguousarray(index, dtype=np.int32)
    s = shading(sh, attr.shape[1], tex)

    def band(rows):
        gs = np.zeros((V, 3))
        ga = np.zeros((V, attr.shape[1])) if want_attr else None
        counts = np.zeros(6, np.int64)
        gabs = np.zeros((V, 3)) if want_abs else None
        gaabs = np.zeros((V, attr.shape[1])) if (want_abs and want_attr) else None
        rc = lib().orc_backward_rows(_p(scr), _p(snap), _p(flags), V, _p(tris_c), _p(index_c), H, W, _p(image),
                                     _p(grad_image), _p(attr), _p(tex), ctypes.byref(s), mode, _p(gs), _p(ga),
                                     _p(counts), _p(gabs), _p(gaabs), rows[0], rows[1])
        assert rc == 0
        return gs, ga, counts, gabs, gaabs

    bands = _bands(H, threads)
    if len(bands) == 1:
        parts = [band(bands[0])]
    else:
        with _pool(len(bands)) as ex:
            parts = list(ex.map(band, bands))
    gs, ga, counts, gabs, gaabs = parts[0]
    for p in parts[1:]:
        gs += p[0]
        if want_attr:
            ga += p[1]
        counts += p[2]
        if want_abs:
            gabs += p[3]
            if want_attr:
                gaabs += p[4]
    names = ["differing", "overhang", "adjacent", "intersection", "intersection_parallel", "intersection_off"]
    if want_abs:
        cnt = dict(zip(names, counts.tolist()))
        cnt["grad_attr_abs"] = gaabs
        return gs, ga, cnt, gabs
    return gs, ga, dict(zip(names, counts.tolist()))


FP32_ULP, FP64_ULP = 2.0 ** -24, 2.0 ** -40


def texel_ambiguity(scr, tris, index, attr, sh, tex, ulp: float = FP32_ULP):
    """Pixels whose texel coordinate is within the error bound of a cell boundary ([H,W] bool): ``ulp`` is the
    unit roundoff of the evaluation compared against (FP32_ULP, or FP64_ULP for FP64 arithmetic)."""
    H, W = index.shape
    out = np.zeros((H, W), np.uint8)
    if sh.uv_offset < 0 or tex is None:
        return out.astype(bool)
    attr = np.ascontiguousarray(attr, dtype=np.float32)
    s = shading(sh, attr.shape[1], tex)
    lib().orc_texel_ambiguity(_p(scr), _p(np.ascontiguousarray(tris, dtype=np.int32)),
                              _p(np.ascontiguousarray(index, dtype=np.int32)), H, W, _p(attr), ctypes.byref(s),
                              float(ulp), _p(out))
    return out.astype(bool)


def forward_grad(scr, snap, flags, tris, index, image, tangent, attr, sh, tex=None,
                 mode: int = EDGE | INTERIOR | INTERSECT, want_abs: bool = False):
    """Forward gradient image [H,W,C] f64 for the projected-vertex tangent [V,3] (+ the magnitude image)."""
    H, W = index.shape
    attr = np.ascontiguousarray(attr, dtype=np.float32)
    tex = None if tex is None else np.ascontiguousarray(tex, dtype=np.float32)
    image = np.ascontiguousarray(image, dtype=np.float64)
    s = shading(sh, attr.shape[1], tex)
    out = np.zeros((H, W, sh.C))
    mag = np.zeros((H, W, sh.C)) if want_abs else None
    rc = lib().orc_forward_grad(_p(scr), _p(np.ascontiguousarray(snap, dtype=np.int64)),
                                _p(np.ascontiguousarray(flags, dtype=np.int32)), len(scr),
                                _p(np.ascontiguousarray(tris, dtype=np.int32)),
                                _p(np.ascontiguousarray(index, dtype=np.int32)), H, W, _p(image), _p(attr), _p(tex),
                                ctypes.byref(s), mode, _p(np.ascontiguousarray(tangent, dtype=np.float64)), _p(out),
                                _p(mag))
    assert rc == 0
    return (out, mag) if want_abs else out


def crossing_weights(scr, snap, tri, f, o, axis):
    """Exact-crossing weights of one overhang pair: foreground pixel f = (x, y), other pixel o; ->
    (vertex ids [2], weights [2]) or None."""
    v = np.zeros(2, np.int32)
    w = np.zeros(2)
    ok = lib().orc_crossing_weights(_p(np.ascontiguousarray(scr, dtype=np.float64)),
                                    _p(np.ascontiguousarray(snap, dtype=np.int64)),
                                    _p(np.ascontiguousarray(tri, dtype=np.int32)), f[0], f[1], o[0], o[1], axis,
                                    _p(v), _p(w))
    return (v, w) if ok else None


def project_jvp(verts, cam, tangent_world):
    verts = np.ascontiguousarray(verts, dtype=np.float32)
    c = camera(cam)
    out = np.zeros((len(verts), 3))
    lib().orc_project_jvp(_p(verts), len(verts), ctypes.byref(c),
                          _p(np.ascontiguousarray(tangent_world, dtype=np.float64)), _p(out))
    return out


def project_backward(verts, cam, grad_scr):
    verts = np.ascontiguousarray(verts, dtype=np.float32)
    out = np.zeros((len(verts), 3))
    c = camera(cam)
    lib().orc_project_backward(_p(verts), len(verts), ctypes.byref(c),
                               _p(np.ascontiguousarray(grad_scr, dtype=np.float64)), _p(out))
    return out


# ---------------------------------------------------------------------------
# whole scenes (all views), thread pool over views
# ---------------------------------------------------------------------------

class ViewResult:
    __slots__ = ("scr", "snap", "flags", "index", "tie", "lam", "bary", "depth", "image", "texamb", "texamb64")


def render_view(verts, tris, cam, H, W, attr, sh, tex=None, threads: int | None = None) -> ViewResult:
    r = ViewResult()
    r.scr, r.snap, r.flags = project(verts, cam)
    r.index, r.tie, _ = rasterize(r.scr, r.snap, r.flags, tris, H, W)
    r.lam, r.bary, r.depth = pixel_values(r.scr, tris, r.index)
    r.image = shade(r.scr, tris, r.index, attr, sh, tex, r.snap, threads=threads)
    r.texamb = texel_ambiguity(r.scr, tris, r.index, attr, sh, tex)
    r.texamb64 = texel_ambiguity(r.scr, tris, r.index, attr, sh, tex, FP64_ULP)
    return r


def _pool(threads: int | None):
    return ThreadPoolExecutor(max_workers=threads or os.cpu_count() or 1)


def render(scene, views=None, threads: int | None = None) -> list[ViewResult]:
    views = range(scene.n_views) if views is None else views
    with _pool(threads) as ex:
        return list(ex.map(lambda i: render_view(scene.verts, scene.tris, scene.cams[i], scene.H, scene.W,
                                                 scene.attr, scene.shading, scene.tex), views))


def backward_scene(scene, results: list[ViewResult], grad_images, views=None,
                   mode: int = EDGE | INTERIOR | INTERSECT, threads: int | None = None, want_attr=False,
                   images=None):
    """Per-view grad_scr list, summed world grad_verts [V,3], per-view counts (and grad_attr).  ``images``: the
    images passed through the edge step, one per view (default: each view's own rendered image)."""
    views = list(range(scene.n_views) if views is None else views)

    def one(k):
        i = views[k]
        r = results[k]
        img = r.image if images is None else images[k]
        gs, ga, cnt, gabs = backward(r.scr, r.snap, r.flags, scene.tris, r.index, img, grad_images[k],
                                     scene.attr, scene.shading, scene.tex, mode, want_attr, want_abs=True)
        gw = project_backward(scene.verts, scene.cams[i], gs)
        cnt["grad_abs"] = gabs
        return gs, ga, gw, cnt

    with _pool(threads) as ex:
        outs = list(ex.map(one, range(len(views))))
    grad_verts = np.zeros((len(scene.verts), 3))
    for o in outs:
        grad_verts += o[2]
    grad_attr = None
    if want_attr:
        grad_attr = sum(o[1] for o in outs)
    return [o[0] for o in outs], grad_verts, [o[3] for o in outs], grad_attr


def world_condition(scene, views, results, S_views):
    """Conditioning sums of the world-space gradients: the per-view sums of |contribution| pushed
    through |R^T J^T| (J = d(x_s, y_s, zeta)/d(X_c, Y_c, Z_c) at the oracle's projection)."""
    Sw = np.zeros((len(scene.verts), 3))
    for k, v in enumerate(views):
        cam = scene.cams[v]
        R = np.asarray(cam["R"], np.float64).reshape(3, 3)
        scr = results[k].scr
        z = scr[:, 2]
        J = np.zeros((len(z), 3, 3))
        J[:, 0, 0] = float(cam["fx"]) * z
        J[:, 0, 2] = -(scr[:, 0] - float(cam["cx"])) * z
        J[:, 1, 1] = float(cam["fy"]) * z
        J[:, 1, 2] = -(scr[:, 1] - float(cam["cy"])) * z
        J[:, 2, 2] = -z * z
        M = np.abs(np.einsum("ji,vkj->vik", R, J))
        Sw += np.einsum("vik,vk->vi", M, S_views[k])
    return Sw
