"""FP64 oracle of the Laplacian preconditioning of vertex updates (Nicolet et al., "Large Steps in Inverse
Rendering of Geometry", 2021), which the paper applies to every mesh optimisation (Sec. 5, Supp. B: lambda 8 to
32, mostly 16).  TEST INFRASTRUCTURE: only ``tests/`` and the benchmark's CPU legs use it.

Definitions written out plainly:

* the edge graph of a triangle mesh: vertices i, j are neighbours iff some triangle has both (i != j);
* the combinatorial Laplacian L = D - A (D the neighbour counts, A the adjacency matrix);
* the reparameterisation u = M x with M = I + lambda L; the gradient with respect to u is M^-1 dL/dx
  (M is symmetric) and the positions are x = M^-1 u;
* the optimiser: Adam whose per-entry second-moment denominator is replaced by its largest value over the
  parameter block (Nicolet et al.'s uniform Adam), here one block per mesh.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def edge_pairs(tris: np.ndarray) -> np.ndarray:
    """Sorted unique undirected edges (i < j) of the triangles, [E, 2] int64."""
    t = np.asarray(tris, dtype=np.int64).reshape(-1, 3)
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    e = e[e[:, 0] != e[:, 1]]
    e = np.sort(e, axis=1)
    return np.unique(e, axis=0)


def laplacian(tris: np.ndarray, V: int) -> sp.csr_matrix:
    """Combinatorial Laplacian D - A of the edge graph, V x V, FP64."""
    e = edge_pairs(tris)
    i = np.concatenate([e[:, 0], e[:, 1]])
    j = np.concatenate([e[:, 1], e[:, 0]])
    A = sp.csr_matrix((np.ones(len(i)), (i, j)), shape=(V, V))
    deg = np.asarray(A.sum(axis=1)).ravel()
    return (sp.diags(deg) - A).tocsr()


def system(tris: np.ndarray, V: int, lam: float) -> sp.csc_matrix:
    """M = I + lambda L."""
    return (sp.identity(V, format="csr") + lam * laplacian(tris, V)).tocsc()


def apply(tris: np.ndarray, V: int, lam: float, x: np.ndarray) -> np.ndarray:
    return system(tris, V, lam) @ np.asarray(x, dtype=np.float64)


def solve(tris: np.ndarray, V: int, lam: float, b: np.ndarray) -> np.ndarray:
    """M^-1 b by a sparse direct solve, columns independently."""
    M = system(tris, V, lam)
    b = np.asarray(b, dtype=np.float64)
    lu = spla.splu(M)
    return np.stack([lu.solve(b[:, c]) for c in range(b.shape[1])], axis=1)


class UniformAdam:
    """Adam on a [V, 3] parameter with one denominator per block of rows: the largest bias-corrected
    second-moment square root in the block (Nicolet et al.).  ``blocks`` are (start, stop) row ranges."""

    def __init__(self, shape, blocks, lr: float, betas=(0.9, 0.999), eps: float = 1e-8):
        self.m = np.zeros(shape)
        self.v = np.zeros(shape)
        self.blocks = list(blocks)
        self.lr, self.b1, self.b2, self.eps = lr, betas[0], betas[1], eps
        self.t = 0

    def step(self, param: np.ndarray, grad: np.ndarray) -> np.ndarray:
        self.t += 1
        self.m = self.b1 * self.m + (1.0 - self.b1) * grad
        self.v = self.b2 * self.v + (1.0 - self.b2) * grad * grad
        mh = self.m / (1.0 - self.b1 ** self.t)
        vh = self.v / (1.0 - self.b2 ** self.t)
        out = param.copy()
        for a, b in self.blocks:
            den = np.sqrt(vh[a:b]).max() + self.eps if b > a else 1.0
            out[a:b] = param[a:b] - self.lr * mh[a:b] / den
        return out
