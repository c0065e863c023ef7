"""ctypes binding of ``libmer.so``: one Python function per C entry point, same names.

Argument marshalling only: tensors are passed as raw device pointers on the
current PyTorch stream; every step of the computation runs in the library's
CUDA kernels.  There is no CPU fallback: without the compiled library (or
without a GPU) these functions raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

MER_OK, MER_EINVAL, MER_ECUDA, MER_EOVERFLOW, MER_ERANGE, MER_EFIXED = 0, 1, 2, 3, 4, 5
MER_EDGE, MER_INTERIOR, MER_INTERSECT, MER_EXACT_CROSSING, MER_DETERMINISTIC = 1, 2, 4, 8, 16
CAMERA_DOUBLES = 17   # mer_camera: R[9], t[3], fx, fy, cx, cy, znear
VERTEX_FLOATS = 8     # mer_vertex: 32 bytes


class MerError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {strerror(code)} (code {code})")
        self.code = code


class MerShading(ctypes.Structure):
    _fields_ = [("n_main", ctypes.c_int), ("C", ctypes.c_int), ("uv_offset", ctypes.c_int),
                ("mask_ch", ctypes.c_int), ("depth_ch", ctypes.c_int), ("C_attr", ctypes.c_int),
                ("tex_h", ctypes.c_int), ("tex_w", ctypes.c_int), ("tex_c", ctypes.c_int),
                ("backface_ch", ctypes.c_int), ("precise", ctypes.c_int)]


class MerItem(ctypes.Structure):
    _fields_ = [("V", ctypes.c_int), ("T", ctypes.c_int), ("H", ctypes.c_int), ("W", ctypes.c_int),
                ("cam", ctypes.c_int), ("pad", ctypes.c_int), ("vert", ctypes.c_int64), ("tri", ctypes.c_int64),
                ("vrec", ctypes.c_int64), ("trec", ctypes.c_int64), ("pix", ctypes.c_int64),
                ("tile", ctypes.c_int64), ("btile", ctypes.c_int64)]


class MerBatchTotals(ctypes.Structure):
    _fields_ = [("vrecs", ctypes.c_int64), ("trecs", ctypes.c_int64), ("pixels", ctypes.c_int64),
                ("tiles", ctypes.c_int64), ("btiles", ctypes.c_int64), ("n_items", ctypes.c_int),
                ("tile", ctypes.c_int), ("mesh_rows", ctypes.c_int64), ("max_tri_density", ctypes.c_double)]


# (name, argtypes, restype); P = pointer, I = int, Z = size_t, L = int64
_P, _I, _Z, _L = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_int64
_SIGS = {
    "mer_strerror": ([_I], ctypes.c_char_p),
    "mer_version": ([], _I),
    "mer_workspace_size": ([_I, _I, _I, _I, _I, _I, _L], _Z),
    "mer_project": ([_P, _I, _P, _I, _P, _P], _I),
    "mer_project_screen": ([_P, _I, _I, _P, _P], _I),
    "mer_rasterize": ([_P, _I, _P, _I, _I, _I, _I, _I, _P, _Z, _P, _P, _P, _P, _P], _I),
    "mer_shade": ([_P, _I, _P, _I, _I, _I, _I, _P, _P, _P, _P, ctypes.POINTER(MerShading), _P, _P, _P], _I),
    "mer_backward_workspace_size": ([_L, _L, _I, _I], _Z),
    "mer_backward": ([_P, _I, _P, _I, _I, _I, _I, _P, _P, _P, _P, _P, _P, ctypes.POINTER(MerShading), _I, _P, _P,
                      _P, _Z, _P], _I),
    "mer_edge_grad_backward": ([_P, _P, _I, _P, _P, _I, _P, _I, _I, _I, _I, _I, _P, _P, _P], _I),
    "mer_interpolate_backward": ([_P, _I, _P, _I, _P, _I, _P, _I, _I, _I, _P, _P, _P, _P, _P], _I),
    "mer_project_backward": ([_I, _P, _I, _P, _P, _P, _P], _I),
    "mer_sync_status": ([_P, ctypes.POINTER(ctypes.c_int64), _P], _I),
    "mer_forward_grad": ([_P, _I, _P, _I, _I, _I, _I, _P, _P, _P, _P, _P, ctypes.POINTER(MerShading), _I, _P, _P,
                          _P], _I),
    "mer_project_jvp": ([_P, _I, _P, _I, _P, _P, _P], _I),
    "mer_vertex_normals": ([_P, _I, _P, ctypes.c_int64, _P, _P, _P, _P], _I),
    "mer_vertex_normals_backward": ([_P, _I, _P, ctypes.c_int64, _P, _P, _P, _P, _P], _I),
    "mer_l2_loss_grad": ([_P, _P, ctypes.c_int64, _P, _P, _P], _I),
    "mer_rasterize_world": ([_P, _I, _P, _I, _P, _I, _I, _I, _I, _P, _Z, _P, _P, _P, _P, _P], _I),
    "mer_laplacian_csr": ([_P, ctypes.c_int64, ctypes.c_int64, _P, _P], _I),
    "mer_precond_apply": ([_P, _P, ctypes.c_int64, ctypes.c_float, _P, _P, _P], _I),
    "mer_precond_solve_workspace_size": ([ctypes.c_int64], _Z),
    "mer_precond_solve": ([_P, _P, ctypes.c_int64, ctypes.c_float, _P, _P, _I, ctypes.c_float, _P, _Z, _P], _I),
    "mer_precond_solve_info": ([_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), _P], _I),
    "mer_rasterize_noalloc": ([_P, _I, _P, _I, _I, _I, _I, _I, _P, _P, _P, _P, _P], _I),
    "mer_batch_plan": ([_P, _I, _I, ctypes.POINTER(MerBatchTotals)], _I),
    "mer_batch_workspace_size": ([ctypes.POINTER(MerBatchTotals), _L], _Z),
    "mer_batch_project": ([_P, _P, _P, ctypes.POINTER(MerBatchTotals), _P, _P], _I),
    "mer_batch_rasterize": ([_P, _P, _P, ctypes.POINTER(MerBatchTotals), _P, _Z, _P, _P, _P, _P, _I, _P], _I),
    "mer_batch_shade": ([_P, _P, _P, ctypes.POINTER(MerBatchTotals), _P, _P, _P, _P, ctypes.POINTER(MerShading), _P,
                         _P, _P], _I),
    "mer_batch_render": ([_P, _P, _P, ctypes.POINTER(MerBatchTotals), _P, _Z, _P, _P, _P, _P, _P, _P, _P,
                          ctypes.POINTER(MerShading), _P, _I, _P], _I),
    "mer_batch_backward": ([_P, _P, _P, ctypes.POINTER(MerBatchTotals), _P, _P, _P, _P, _P, _P,
                            ctypes.POINTER(MerShading), _I, _P, _P, _P, _Z, _I, _P], _I),
    "mer_batch_project_backward": ([_P, _P, ctypes.POINTER(MerBatchTotals), _P, _P, _P, _P, _Z, _P], _I),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libmer.so (building it first if it is missing or stale and nvcc is available)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if build_if_missing:
            try:
                path = _build.build_lib()
            except RuntimeError:
                if not os.path.exists(path):
                    raise
        if not os.path.exists(path):
            raise RuntimeError(f"libmer.so is not built ({path}); run paper_2405_02508_gb300.build.build_lib()")
        L = ctypes.CDLL(path)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


def strerror(code: int) -> str:
    return lib().mer_strerror(code).decode()


def _check(code: int, where: str):
    if code != MER_OK:
        raise MerError(code, where)


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libmer takes device tensors")
    if not t.is_contiguous():
        raise ValueError("libmer takes contiguous tensors")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _nbytes(t: torch.Tensor | None) -> int:
    return 0 if t is None else t.numel() * t.element_size()


def shading_struct(sh, C_attr: int, tex: torch.Tensor | None, precise: bool = False) -> MerShading:
    s = MerShading()
    s.n_main, s.C, s.uv_offset, s.mask_ch, s.depth_ch = sh.n_main, sh.C, sh.uv_offset, sh.mask_ch, sh.depth_ch
    s.C_attr = C_attr
    s.tex_h, s.tex_w = (int(tex.shape[0]), int(tex.shape[1])) if tex is not None else (0, 0)
    s.tex_c = int(tex.shape[2]) if tex is not None else 0
    s.backface_ch = getattr(sh, "backface_ch", -1)
    s.precise = int(bool(precise))
    return s


def attr_grad_channels(sh: MerShading, grad_attr) -> int:
    """Channels of grad_attr a backward pass writes (the interpolated ones, or u and v)."""
    if grad_attr is None:
        return 0
    return sh.n_main if sh.uv_offset < 0 else 2


def cameras_tensor(cams: np.ndarray, device="cuda") -> torch.Tensor:
    """Packed mer_camera records [n, 17] float64 on the device."""
    a = np.ascontiguousarray(cams).view(np.float64).reshape(len(cams), CAMERA_DOUBLES)
    return torch.from_numpy(a.copy()).to(device)


# ---------------------------------------------------------------------------
# entry points
# ---------------------------------------------------------------------------

def mer_workspace_size(V: int, T: int, n: int, H: int, W: int, tile: int, bin_capacity: int = 0) -> int:
    return int(lib().mer_workspace_size(V, T, n, H, W, tile, bin_capacity))


def mer_project(verts: torch.Tensor, cams: torch.Tensor, vpix: torch.Tensor):
    V, n = verts.shape[0], cams.shape[0]
    _check(lib().mer_project(_ptr(verts), V, _ptr(cams), n, _ptr(vpix), _stream()), "mer_project")


def mer_project_screen(scr: torch.Tensor, vpix: torch.Tensor):
    n, V = scr.shape[0], scr.shape[1]
    _check(lib().mer_project_screen(_ptr(scr), V, n, _ptr(vpix), _stream()), "mer_project_screen")


def mer_rasterize(vpix, tris, H, W, tile, workspace, index, depth=None, bary=None, cover=None):
    n, V = vpix.shape[0], vpix.shape[1]
    T = tris.shape[0]
    _check(lib().mer_rasterize(_ptr(vpix), V, _ptr(tris), T, n, H, W, tile, _ptr(workspace),
                               workspace.numel() * workspace.element_size(), _ptr(index), _ptr(depth), _ptr(bary),
                               _ptr(cover), _stream()), "mer_rasterize")


def mer_shade(vpix, tris, index, attr, tex, bg: np.ndarray, sh: MerShading, image, status_ws=None):
    n, V = vpix.shape[0], vpix.shape[1]
    H, W = index.shape[1], index.shape[2]
    bgc = (ctypes.c_float * max(1, sh.C))(*[float(x) for x in bg])
    _check(lib().mer_shade(_ptr(vpix), V, _ptr(tris), tris.shape[0], n, H, W, _ptr(index), _ptr(attr), _ptr(tex),
                           ctypes.cast(bgc, ctypes.c_void_p), ctypes.byref(sh), _ptr(image), _ptr(status_ws),
                           _stream()), "mer_shade")


def mer_backward_workspace_size(vertex_rows: int, attr_rows: int, attr_channels: int, terms: int) -> int:
    return int(lib().mer_backward_workspace_size(vertex_rows, attr_rows, attr_channels, terms))


def mer_backward(vpix, tris, index, image, grad_image, attr, tex, sh: MerShading, terms: int, grad_vpix,
                 grad_attr=None, status_ws=None, cover=None):
    """``status_ws``: the workspace (status header; with MER_DETERMINISTIC also the fixed-point sums)."""
    n, V = vpix.shape[0], vpix.shape[1]
    H, W = index.shape[1], index.shape[2]
    _check(lib().mer_backward(_ptr(vpix), V, _ptr(tris), tris.shape[0], n, H, W, _ptr(index), _ptr(cover), _ptr(image),
                              _ptr(grad_image), _ptr(attr), _ptr(tex), ctypes.byref(sh), terms, _ptr(grad_vpix),
                              _ptr(grad_attr), _ptr(status_ws), _nbytes(status_ws), _stream()), "mer_backward")


def mer_edge_grad_backward(image, grad_image, index, vpix, tris, intersections: bool, grad_vpix, status_ws=None):
    n, V = vpix.shape[0], vpix.shape[1]
    H, W, C = image.shape[1], image.shape[2], image.shape[3]
    _check(lib().mer_edge_grad_backward(_ptr(image), _ptr(grad_image), C, _ptr(index), _ptr(vpix), V, _ptr(tris),
                                        tris.shape[0], n, H, W, int(bool(intersections)), _ptr(grad_vpix),
                                        _ptr(status_ws), _stream()), "mer_edge_grad_backward")


def mer_interpolate_backward(attr, tris, vpix, index, grad_out, grad_attr, grad_vpix, status_ws=None):
    n, V = vpix.shape[0], vpix.shape[1]
    H, W = index.shape[1], index.shape[2]
    _check(lib().mer_interpolate_backward(_ptr(attr), attr.shape[1], _ptr(tris), tris.shape[0], _ptr(vpix), V,
                                          _ptr(index), n, H, W, _ptr(grad_out), _ptr(grad_attr), _ptr(grad_vpix),
                                          _ptr(status_ws), _stream()), "mer_interpolate_backward")


def mer_project_backward(cams, vpix, grad_vpix, grad_verts):
    n, V = vpix.shape[0], vpix.shape[1]
    _check(lib().mer_project_backward(V, _ptr(cams), n, _ptr(vpix), _ptr(grad_vpix), _ptr(grad_verts), _stream()),
           "mer_project_backward")


def mer_sync_status(workspace) -> tuple[int, int]:
    tot = ctypes.c_int64(0)
    code = lib().mer_sync_status(_ptr(workspace), ctypes.byref(tot), _stream())
    return code, int(tot.value)


def mer_forward_grad(vpix, tris, index, image, tangent, attr, tex, sh: MerShading, terms: int, out, status_ws=None):
    n, V = vpix.shape[0], vpix.shape[1]
    H, W = index.shape[1], index.shape[2]
    _check(lib().mer_forward_grad(_ptr(vpix), V, _ptr(tris), tris.shape[0], n, H, W, _ptr(index), _ptr(image),
                                  _ptr(tangent), _ptr(attr), _ptr(tex), ctypes.byref(sh), terms, _ptr(out),
                                  _ptr(status_ws), _stream()), "mer_forward_grad")


def mer_project_jvp(tangent_world, cams, vpix, out):
    n, V = vpix.shape[0], vpix.shape[1]
    _check(lib().mer_project_jvp(_ptr(tangent_world), V, _ptr(cams), n, _ptr(vpix), _ptr(out), _stream()),
           "mer_project_jvp")


def mer_vertex_normals(verts, tris, acc, normals, status_ws=None):
    _check(lib().mer_vertex_normals(_ptr(verts), verts.shape[0], _ptr(tris), tris.shape[0], _ptr(acc), _ptr(normals),
                                    _ptr(status_ws), _stream()), "mer_vertex_normals")


def mer_vertex_normals_backward(verts, tris, acc, grad_normals, grad_verts, status_ws=None):
    _check(lib().mer_vertex_normals_backward(_ptr(verts), verts.shape[0], _ptr(tris), tris.shape[0], _ptr(acc),
                                             _ptr(grad_normals), _ptr(grad_verts), _ptr(status_ws), _stream()),
           "mer_vertex_normals_backward")


def mer_l2_loss_grad(image, target, grad, loss):
    _check(lib().mer_l2_loss_grad(_ptr(image), _ptr(target), image.numel(), _ptr(grad), _ptr(loss), _stream()),
           "mer_l2_loss_grad")


def mer_rasterize_world(verts, tris, cams, H, W, tile, workspace, index, vpix, depth=None, bary=None):
    n, V = vpix.shape[0], vpix.shape[1]
    _check(lib().mer_rasterize_world(_ptr(verts), V, _ptr(tris), tris.shape[0], _ptr(cams), n, H, W, tile,
                                     _ptr(workspace), workspace.numel() * workspace.element_size(), _ptr(index),
                                     _ptr(depth), _ptr(bary), _ptr(vpix), _stream()), "mer_rasterize_world")


def mer_laplacian_csr(tris: np.ndarray, V: int) -> tuple[np.ndarray, np.ndarray]:
    """Host call: (row_ptr [V+1] int64, col [nnz] int32) of the meshes' edge graph."""
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    row_ptr = np.zeros(V + 1, dtype=np.int64)
    tp = tris.ctypes.data_as(ctypes.c_void_p) if tris.size else None
    _check(lib().mer_laplacian_csr(tp, len(tris), V, row_ptr.ctypes.data_as(ctypes.c_void_p), None),
           "mer_laplacian_csr")
    col = np.zeros(max(int(row_ptr[-1]), 1), dtype=np.int32)
    _check(lib().mer_laplacian_csr(tp, len(tris), V, row_ptr.ctypes.data_as(ctypes.c_void_p),
                                   col.ctypes.data_as(ctypes.c_void_p)), "mer_laplacian_csr")
    return row_ptr, col[: int(row_ptr[-1])]


def mer_precond_apply(row_ptr, col, lam: float, x, y):
    _check(lib().mer_precond_apply(_ptr(row_ptr), _ptr(col), x.shape[0], float(lam), _ptr(x), _ptr(y), _stream()),
           "mer_precond_apply")


def mer_precond_solve(row_ptr, col, lam: float, b, x, max_iters: int, rel_tol: float, workspace):
    _check(lib().mer_precond_solve(_ptr(row_ptr), _ptr(col), b.shape[0], float(lam), _ptr(b), _ptr(x), max_iters,
                                   float(rel_tol), _ptr(workspace), workspace.numel() * workspace.element_size(),
                                   _stream()), "mer_precond_solve")


def mer_precond_solve_info(workspace) -> tuple[int, float]:
    it = ctypes.c_int(0)
    res = ctypes.c_double(0.0)
    _check(lib().mer_precond_solve_info(_ptr(workspace), ctypes.byref(it), ctypes.byref(res), _stream()),
           "mer_precond_solve_info")
    return int(it.value), float(res.value)


def mer_rasterize_noalloc(vpix, tris, H, W, tile, index, depth=None, bary=None, status=None):
    """mer_rasterize with the library's own fixed workspace (no device allocation by anyone at call time).
    ``status``: optional device int32 tensor of one element receiving the status bits."""
    n, V = vpix.shape[0], vpix.shape[1]
    _check(lib().mer_rasterize_noalloc(_ptr(vpix), V, _ptr(tris), tris.shape[0], n, H, W, tile, _ptr(index),
                                       _ptr(depth), _ptr(bary), _ptr(status), _stream()), "mer_rasterize_noalloc")


# ---------------------------------------------------------------------------
# batched path
# ---------------------------------------------------------------------------

def mer_batch_plan(items, tile: int) -> MerBatchTotals:
    """items: ctypes array of MerItem (host); fills the offsets in place and returns the totals."""
    tot = MerBatchTotals()
    _check(lib().mer_batch_plan(ctypes.cast(items, ctypes.c_void_p), len(items), tile, ctypes.byref(tot)),
           "mer_batch_plan")
    return tot


def mer_batch_workspace_size(tot: MerBatchTotals, bin_capacity: int = 0) -> int:
    return int(lib().mer_batch_workspace_size(ctypes.byref(tot), bin_capacity))


def mer_batch_project(verts, cams, items_dev, tot, vpix):
    _check(lib().mer_batch_project(_ptr(verts), _ptr(cams), _ptr(items_dev), ctypes.byref(tot), _ptr(vpix), _stream()),
           "mer_batch_project")


def mer_batch_rasterize(vpix, tris, items_dev, tot, workspace, index, depth=None, bary=None, persistent_ctas=0,
                        cover=None):
    _check(lib().mer_batch_rasterize(_ptr(vpix), _ptr(tris), _ptr(items_dev), ctypes.byref(tot), _ptr(workspace),
                                     workspace.numel() * workspace.element_size(), _ptr(index), _ptr(depth),
                                     _ptr(bary), _ptr(cover), persistent_ctas, _stream()), "mer_batch_rasterize")


def mer_batch_shade(vpix, tris, items_dev, tot, index, attr, tex, bg, sh: MerShading, image, status_ws=None):
    bgc = (ctypes.c_float * max(1, sh.C))(*[float(x) for x in bg])
    _check(lib().mer_batch_shade(_ptr(vpix), _ptr(tris), _ptr(items_dev), ctypes.byref(tot), _ptr(index), _ptr(attr),
                                 _ptr(tex), ctypes.cast(bgc, ctypes.c_void_p), ctypes.byref(sh), _ptr(image),
                                 _ptr(status_ws), _stream()), "mer_batch_shade")


def mer_batch_render(vpix, tris, items_dev, tot, workspace, index, attr, tex, bg, sh: MerShading, image, depth=None,
                     bary=None, persistent_ctas=0, cover=None):
    bgc = (ctypes.c_float * max(1, sh.C))(*[float(x) for x in bg])
    _check(lib().mer_batch_render(_ptr(vpix), _ptr(tris), _ptr(items_dev), ctypes.byref(tot), _ptr(workspace),
                                  workspace.numel() * workspace.element_size(), _ptr(index), _ptr(depth), _ptr(bary),
                                  _ptr(cover), _ptr(attr), _ptr(tex), ctypes.cast(bgc, ctypes.c_void_p), ctypes.byref(sh),
                                  _ptr(image), persistent_ctas, _stream()), "mer_batch_render")


def mer_batch_backward(vpix, tris, items_dev, tot, index, image, grad_image, attr, tex, sh: MerShading, terms: int,
                       grad_vpix, grad_attr, workspace, persistent_ctas=0, cover=None):
    _check(lib().mer_batch_backward(_ptr(vpix), _ptr(tris), _ptr(items_dev), ctypes.byref(tot), _ptr(index),
                                    _ptr(cover), _ptr(image), _ptr(grad_image), _ptr(attr), _ptr(tex), ctypes.byref(sh), terms,
                                    _ptr(grad_vpix), _ptr(grad_attr), _ptr(workspace), _nbytes(workspace),
                                    persistent_ctas, _stream()),
           "mer_batch_backward")


def mer_batch_project_backward(cams, items_dev, tot, vpix, grad_vpix, grad_verts, workspace=None):
    """workspace: None for the FP32 atomic path; a workspace tensor for the reproducible FP64 path."""
    _check(lib().mer_batch_project_backward(_ptr(cams), _ptr(items_dev), ctypes.byref(tot), _ptr(vpix),
                                            _ptr(grad_vpix), _ptr(grad_verts), _ptr(workspace), _nbytes(workspace),
                                            _stream()),
           "mer_batch_project_backward")
