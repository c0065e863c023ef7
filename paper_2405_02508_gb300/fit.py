"""Inverse rendering over an uneven batch of meshes: fit perturbed vertex positions to images rendered from
the unperturbed meshes (mask + normal L2), with Adam.

``BatchRender`` is the autograd function of the batched path: forward renders every item, backward runs
the micro-edge + interior kernels and returns d(loss)/d(vertices) and d(loss)/d(attributes).  Vertex
normals (the attributes) are recomputed from the current positions with PyTorch each step, so the
attribute gradient reaches the positions through PyTorch's own autograd.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B
from .batch import BatchRenderer


class BatchRender(torch.autograd.Function):
    """image [pixels, C] = render(verts, attr).  The renderer keeps the forward image for the backward, so
    call backward before the next forward on the same renderer."""

    @staticmethod
    def forward(ctx, verts, attr, br: BatchRenderer):
        br.forward(verts.contiguous(), attr.contiguous())
        ctx.br = br
        ctx.save_for_backward(attr)
        return br.image.clone()

    @staticmethod
    def backward(ctx, grad_image):
        (attr,) = ctx.saved_tensors
        br = ctx.br
        ga = torch.zeros_like(attr) if ctx.needs_input_grad[1] else None
        gv = br.backward(grad_image.contiguous(), attr, None, grad_attr=ga)
        return gv.clone(), ga, None


class VertexNormals(torch.autograd.Function):
    """Area-weighted, normalised vertex normals on the device (mer_vertex_normals and its backward)."""

    @staticmethod
    def forward(ctx, verts, tris32):
        verts = verts.contiguous()
        acc = torch.empty_like(verts)
        nrm = torch.empty_like(verts)
        B.mer_vertex_normals(verts, tris32, acc, nrm)
        ctx.save_for_backward(verts, tris32, acc)
        return nrm

    @staticmethod
    def backward(ctx, grad_n):
        verts, tris32, acc = ctx.saved_tensors
        g = grad_n.contiguous().clone()
        gv = torch.zeros_like(verts)
        B.mer_vertex_normals_backward(verts, tris32, acc, g, gv)
        return gv, None


def vertex_normals(verts: torch.Tensor, tris: torch.Tensor) -> torch.Tensor:
    """Area-weighted, normalised vertex normals (differentiable, PyTorch)."""
    a, b, c = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    fn = torch.cross(b - a, c - a, dim=1)
    vn = torch.zeros_like(verts).index_add_(0, tris[:, 0], fn).index_add_(0, tris[:, 1], fn).index_add_(0, tris[:, 2], fn)
    return vn / vn.norm(dim=1, keepdim=True).clamp_min(1e-20)


class UnevenFit:
    """The uneven-batch fitting problem on the GPU batched path."""

    def __init__(self, items, sigma: float = 0.01, seed: int = 11, tile: int = 32):
        self.items = items
        meshes = [(it.verts, it.tris) for it in items]
        cams = np.concatenate([it.cams for it in items])
        self.br = BatchRenderer(meshes, [(k, k, it.H, it.W) for k, it in enumerate(items)], cams,
                                items[0].shading, 3, None, tile=tile)
        off = np.cumsum([0] + [len(it.verts) for it in items])
        self.vert_off = off
        self.tris_global = torch.from_numpy(np.concatenate([it.tris + off[k] for k, it in enumerate(items)])).long().cuda()
        self.tris32 = self.tris_global.int().contiguous()
        self.v_true = torch.from_numpy(np.concatenate([it.verts for it in items])).cuda()
        rng = np.random.default_rng(seed)
        self.v_init = self.v_true + torch.from_numpy(rng.normal(0.0, sigma, self.v_true.shape).astype(np.float32)).cuda()
        with torch.no_grad():
            self.br.prepare(self.v_true, self.normals(self.v_true))
            self.target = self.br.image.clone()

    def normals(self, x: torch.Tensor) -> torch.Tensor:
        """Vertex normals of all meshes at positions x (device kernels, differentiable)."""
        return VertexNormals.apply(x, self.tris32)

    @property
    def pixels(self) -> int:
        return int(self.br.tot.pixels)

    @torch.no_grad()
    def loss(self, x: torch.Tensor) -> float:
        """The mask + normal L2 loss at positions x."""
        self._render(x.contiguous())
        self._l2()
        return float(self._loss.item())

    def _render(self, x: torch.Tensor) -> torch.Tensor:
        """Normals (kept for the backward) and the batched render at positions x; returns the normals."""
        if getattr(self, "_nacc", None) is None or self._nacc.shape != x.shape:
            self._nacc = torch.empty_like(x)
            self._nrm = torch.empty_like(x)
            self._gimg = torch.empty_like(self.target)
            self._loss = torch.zeros(1, dtype=torch.float64, device=x.device)
        B.mer_vertex_normals(x, self.tris32, self._nacc, self._nrm)
        self.br.forward(x, self._nrm)
        return self._nrm

    def _l2(self):
        self._loss.zero_()
        B.mer_l2_loss_grad(self.br.image, self.target, self._gimg, self._loss)

    @torch.no_grad()
    def loss_grad(self, x: torch.Tensor) -> torch.Tensor:
        """dL/dx of the mask + normal L2 loss at positions x, all in device kernels: normals, render, the loss
        gradient, the micro-edge + interior backward (positions and normals), the normals' backward.  The
        returned tensor is the renderer's buffer, valid until the next call."""
        x = x.contiguous()
        nrm = self._render(x)
        self._l2()
        ga = torch.zeros_like(nrm)
        gv = self.br.backward(self._gimg, nrm, grad_attr=ga)
        B.mer_vertex_normals_backward(x, self.tris32, self._nacc, ga, gv)
        return gv

    def run(self, steps: int, lr: float = 1e-3):
        """Plain per-vertex Adam on the positions."""
        verts = self.v_init.clone().requires_grad_(True)
        opt = torch.optim.Adam([verts], lr=lr)
        for _ in range(steps):
            verts.grad = self.loss_grad(verts.detach())
            opt.step()
        return verts.detach()

    def run_preconditioned(self, steps: int, lr: float = 1e-2, lam: float = 16.0, x0: torch.Tensor | None = None):
        """Large-steps loop: uniform Adam on u = (I + lam L) x, gradients and positions through the device
        solves (both warm-started)."""
        from .precond import LaplacianPreconditioner, UniformAdam

        if getattr(self, "_precond", None) is None or self._precond.lam != lam:
            tris = self.tris_global.cpu().numpy().astype(np.int32)
            self._precond = LaplacianPreconditioner(tris, len(self.v_true), lam)
            block = np.concatenate([np.full(self.vert_off[k + 1] - self.vert_off[k], k)
                                    for k in range(len(self.items))])
            self._block = torch.from_numpy(block).cuda()
        P = self._precond
        x = (self.v_init if x0 is None else x0).clone()
        u = P.apply(x)
        opt = UniformAdam(u, self._block, len(self.items), lr)
        gu = torch.zeros_like(x)
        for _ in range(steps):
            gu = P.solve(self.loss_grad(x), gu)
            opt.step(gu)
            x = P.solve(u, x)
        return x

    def rmse(self, verts, subset=None) -> float:
        d = (verts - self.v_true).double()
        if subset is not None:
            rows = np.concatenate([np.arange(self.vert_off[k], self.vert_off[k + 1]) for k in subset])
            d = d[torch.from_numpy(rows).cuda()]
        return float(d.pow(2).sum(dim=1).mean().sqrt())
