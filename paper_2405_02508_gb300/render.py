"""Forward/backward calls over the C-ABI, and the ``torch.autograd.Function``.

``Renderer`` owns the caller-side buffers (workspace, vertex records, images)
for one mesh and a batch of views and chains the library calls:

    forward : mer_project -> mer_rasterize -> mer_shade
    backward: mer_backward (edge + interior) -> mer_project_backward

With ``cover_hint`` (default) the rasterizer also writes the cover image (which facings cover each pixel
centre, one byte a pixel) and the backward uses it to skip pixel pairs that cannot scatter; the results are
the same without it.

``MerRender.apply(verts, attr, tex, cams, renderer, recompute_bary)`` exposes the
same as an autograd function whose backward is the micro-edge kernel (with the
renderer's ``terms``; with MER_DETERMINISTIC among them the gradients are bitwise
reproducible).  With
``recompute_bary`` the barycentric image is never stored (the backward always
re-derives barycentrics from the index image and the vertex records), which
saves 8 bytes per pixel of activation memory.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


class Renderer:
    def __init__(self, tris: torch.Tensor, V: int, n_views: int, H: int, W: int, shading, C_attr: int,
                 tex_shape=None, tile: int = 16, device: str = "cuda", cover_hint: bool = True,
                 precise: bool = False):
        """precise: FP64 shading rounded once per value (the image a MER_DETERMINISTIC backward expects).
        ``terms`` (attribute): the backward terms MerRender uses."""
        self.tris = tris.to(device=device, dtype=torch.int32).contiguous()
        self.T = int(self.tris.shape[0])
        self.V, self.n, self.H, self.W = int(V), int(n_views), int(H), int(W)
        self.tile = tile
        self.device = device
        self.shading = shading
        self.C = shading.C
        self.sh = B.shading_struct(shading, C_attr, None, precise)
        if tex_shape is not None:
            self.sh.tex_h, self.sh.tex_w = int(tex_shape[0]), int(tex_shape[1])
            self.sh.tex_c = int(tex_shape[2]) if len(tex_shape) > 2 else shading.n_main
        self.bg = shading.bg_array()
        n, H, W = self.n, self.H, self.W
        self.vpix = torch.empty((n, self.V, B.VERTEX_FLOATS), dtype=torch.float32, device=device)
        self.index = torch.empty((n, H, W), dtype=torch.int32, device=device)
        self.image = torch.empty((n, H, W, self.C), dtype=torch.float32, device=device)
        self.cover = torch.empty((n, H, W), dtype=torch.uint8, device=device) if cover_hint else None
        self.grad_vpix = torch.zeros((n, self.V, 3), dtype=torch.float64, device=device)
        self.grad_verts = torch.zeros((self.V, 3), dtype=torch.float32, device=device)
        self.terms = B.MER_EDGE | B.MER_INTERIOR | B.MER_INTERSECT
        self._alloc_workspace(0)

    def _alloc_workspace(self, capacity: int, at_least: int = 0):
        nbytes = max(B.mer_workspace_size(self.V, self.T, self.n, self.H, self.W, self.tile, capacity), at_least)
        self.workspace = torch.zeros((nbytes + 255) // 256 * 64, dtype=torch.float32, device=self.device)

    def _ensure_backward_workspace(self, terms: int, grad_attr):
        need = B.mer_backward_workspace_size(self.n * self.V, self.V, B.attr_grad_channels(self.sh, grad_attr), terms)
        if self.workspace.numel() * 4 < need:  # the raster's bins are not needed any more at this point
            self._alloc_workspace(0, need)

    # -- forward -----------------------------------------------------------------------------------
    def project(self, verts: torch.Tensor, cams: torch.Tensor):
        B.mer_project(verts.contiguous(), cams, self.vpix)

    def project_screen(self, scr: torch.Tensor):
        B.mer_project_screen(scr.contiguous(), self.vpix)

    def rasterize(self, depth: torch.Tensor | None = None, bary: torch.Tensor | None = None, checked: bool = True):
        B.mer_rasterize(self.vpix, self.tris, self.H, self.W, self.tile, self.workspace, self.index, depth, bary,
                        self.cover)
        if checked:
            code, total = B.mer_sync_status(self.workspace)
            if code == B.MER_EOVERFLOW:  # size the bin list exactly and redo
                self._alloc_workspace(int(total * 1.25) + 1024)
                B.mer_rasterize(self.vpix, self.tris, self.H, self.W, self.tile, self.workspace, self.index, depth,
                                bary, self.cover)
                code, total = B.mer_sync_status(self.workspace)
            if code != B.MER_OK:
                raise B.MerError(code, "mer_rasterize")

    def shade(self, attr: torch.Tensor, tex: torch.Tensor | None):
        B.mer_shade(self.vpix, self.tris, self.index, attr.contiguous(), tex, self.bg, self.sh, self.image,
                    self.workspace)

    def forward(self, verts, cams, attr, tex=None, depth=None, bary=None, checked=True):
        self.project(verts, cams)
        self.rasterize(depth, bary, checked)
        self.shade(attr, tex)
        return self.image

    # -- backward ----------------------------------------------------------------------------------
    def backward(self, grad_image: torch.Tensor, cams: torch.Tensor, attr: torch.Tensor, tex=None,
                 terms: int = B.MER_EDGE | B.MER_INTERIOR | B.MER_INTERSECT, grad_attr=None, zero: bool = True):
        if zero:
            self.grad_vpix.zero_()
            self.grad_verts.zero_()
        self._ensure_backward_workspace(terms, grad_attr)
        B.mer_backward(self.vpix, self.tris, self.index, self.image, grad_image.contiguous(), attr.contiguous(), tex,
                       self.sh, terms, self.grad_vpix, grad_attr, self.workspace, self.cover)
        B.mer_project_backward(cams, self.vpix, self.grad_vpix, self.grad_verts)
        return self.grad_verts

    # -- forward gradients ---------------------------------------------------------------------------
    def forward_grad(self, tangent_world: torch.Tensor, cams: torch.Tensor, attr: torch.Tensor, tex=None,
                     terms: int = B.MER_EDGE | B.MER_INTERIOR | B.MER_INTERSECT) -> torch.Tensor:
        """d(image)/d(theta) [n,H,W,C] for a world-space vertex tangent [V,3] (after ``forward``)."""
        tv = torch.empty((self.n, self.V, 3), dtype=torch.float32, device=self.device)
        B.mer_project_jvp(tangent_world.contiguous(), cams, self.vpix, tv)
        out = torch.empty_like(self.image)
        B.mer_forward_grad(self.vpix, self.tris, self.index, self.image, tv, attr.contiguous(), tex, self.sh, terms,
                           out, self.workspace)
        return out

    def check_status(self):
        code, _ = B.mer_sync_status(self.workspace)
        if code != B.MER_OK:
            raise B.MerError(code, "device status")


class MerRender(torch.autograd.Function):
    """image = render(verts, attr); backward = micro-edge + interior kernels.

    ``verts`` [V,3] and ``attr`` [V,C_attr] are differentiable; ``tex`` and the
    cameras are not.  The renderer's shading program decides the channels.
    """

    @staticmethod
    def forward(ctx, verts, attr, tex, cams, renderer: Renderer, recompute_bary: bool = True):
        r = renderer
        bary = None
        if not recompute_bary:
            bary = torch.empty((r.n, r.H, r.W, 2), dtype=torch.float32, device=r.device)
        r.forward(verts, cams, attr, tex, bary=bary)
        image = r.image.clone()
        ctx.renderer = r
        ctx.save_for_backward(verts, attr, cams, r.vpix.clone(), r.index.clone(), image,
                              *(() if tex is None else (tex,)), *(() if bary is None else (bary,)))
        ctx.has_tex = tex is not None
        return image

    @staticmethod
    def backward(ctx, grad_image):
        r = ctx.renderer
        saved = ctx.saved_tensors
        verts, attr, cams, vpix, index, image = saved[:6]
        tex = saved[6] if ctx.has_tex else None
        r.vpix.copy_(vpix)
        r.index.copy_(index)
        r.image.copy_(image)
        grad_attr = torch.zeros_like(attr) if ctx.needs_input_grad[1] else None
        gv = r.backward(grad_image, cams, attr, tex, terms=r.terms, grad_attr=grad_attr)
        return gv.clone(), grad_attr, None, None, None, None
