"""Laplacian preconditioning of vertex updates (Nicolet et al., "Large Steps in Inverse Rendering of Geometry",
2021), which the paper uses for all of its mesh optimisations (Sec. 5, Supp. B: lambda 8 to 32, mostly 16).

Positions x [V, 3] are reparameterised as u = M x, M = I + lambda L (L the combinatorial Laplacian of the
meshes' edge graph, one independent block per mesh).  A step takes the gradient with respect to u,
M^-1 dL/dx, updates u with ``UniformAdam`` and maps back with x = M^-1 u.  Both solves are conjugate
gradients in the library's kernels (``mer_precond_solve``), warm-started from the previous step's result.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


class LaplacianPreconditioner:
    def __init__(self, tris: np.ndarray, V: int, lam: float = 16.0, max_iters: int = 200, rel_tol: float = 1e-6,
                 device: str = "cuda"):
        """tris: [T, 3] int32 over all meshes (global vertex ids); V: number of vertex rows."""
        row_ptr, col = B.mer_laplacian_csr(tris, V)
        self.V = V
        self.lam = float(lam)
        self.max_iters = max_iters
        self.rel_tol = rel_tol
        self.row_ptr = torch.from_numpy(row_ptr).to(device)
        self.col = torch.from_numpy(col if len(col) else np.zeros(1, np.int32)).to(device)
        nbytes = B.lib().mer_precond_solve_workspace_size(V)
        self.workspace = torch.zeros((nbytes + 255) // 256 * 64, dtype=torch.float32, device=device)

    def apply(self, x: torch.Tensor) -> torch.Tensor:
        """M x."""
        y = torch.empty_like(x)
        B.mer_precond_apply(self.row_ptr, self.col, self.lam, x.contiguous(), y)
        return y

    def solve(self, b: torch.Tensor, x0: torch.Tensor | None = None) -> torch.Tensor:
        """M^-1 b, starting from x0 (zeros if None)."""
        x = torch.zeros_like(b) if x0 is None else x0.clone()
        B.mer_precond_solve(self.row_ptr, self.col, self.lam, b.contiguous(), x, self.max_iters, self.rel_tol,
                            self.workspace)
        return x

    def last_solve(self) -> tuple[int, float]:
        """(iterations, relative residual) of the last solve (synchronises)."""
        return B.mer_precond_solve_info(self.workspace)


class UniformAdam:
    """Adam on a [V, 3] parameter whose per-entry denominator is replaced by the largest bias-corrected
    second-moment square root of the entry's block (Nicolet et al.'s uniform Adam; one block per mesh, so the
    meshes of a batch stay independent problems)."""

    def __init__(self, param: torch.Tensor, block_of_row: torch.Tensor, n_blocks: int, lr: float,
                 betas=(0.9, 0.999), eps: float = 1e-8):
        self.param = param
        self.block = block_of_row.long()
        self.n_blocks = n_blocks
        self.lr, self.b1, self.b2, self.eps = lr, betas[0], betas[1], eps
        self.m = torch.zeros_like(param)
        self.v = torch.zeros_like(param)
        self.t = 0

    @torch.no_grad()
    def step(self, grad: torch.Tensor):
        self.t += 1
        self.m.mul_(self.b1).add_(grad, alpha=1.0 - self.b1)
        self.v.mul_(self.b2).addcmul_(grad, grad, value=1.0 - self.b2)
        mh = self.m / (1.0 - self.b1 ** self.t)
        vh = self.v / (1.0 - self.b2 ** self.t)
        row = vh.sqrt().amax(dim=1)
        blk = torch.zeros(self.n_blocks, dtype=row.dtype, device=row.device)
        blk.scatter_reduce_(0, self.block, row, reduce="amax", include_self=True)
        self.param.sub_(self.lr * mh / (blk[self.block] + self.eps)[:, None])
