"""The uneven-batch fitting loop driven by the FP64 oracle's gradients.  TEST INFRASTRUCTURE: only the test
suite and the benchmark's CPU-baseline leg use it.

The loop is the one the library's batched path runs (``fit.UnevenFit.run``): the mask + normal L2 loss
against images rendered from the unperturbed meshes, vertex normals recomputed from the current positions
(area-weighted face normals summed at each vertex, normalised), and plain per-vertex Adam on the positions.
Here every item's image, micro-edge + interior gradient (Eq. 11, Sec. 4.3, Eq. 12, Eq. 5) and projection
backward come from oracle.c in FP64, and the normals' derivative from PyTorch autograd in FP64.  Each view's
shading and backward run in bands of rows on ``threads`` threads.
"""
from __future__ import annotations

import os

import numpy as np
import torch

from . import oracle as orc


def vertex_normals_fp64(verts: torch.Tensor, tris: torch.Tensor) -> torch.Tensor:
    """Area-weighted, normalised vertex normals of FP64 positions, differentiable by autograd."""
    a, b, c = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    face = torch.linalg.cross(b - a, c - a, dim=1)
    acc = torch.zeros_like(verts)
    for k in range(3):
        acc = acc.index_add(0, tris[:, k], face)
    return acc / acc.norm(dim=1, keepdim=True).clamp_min(1e-20)


def oracle_fit(items, v_init: np.ndarray, steps: int, lr: float = 1e-3, threads: int | None = None) -> np.ndarray:
    """``steps`` Adam steps from v_init (rows of all items' vertices, in item order) with oracle gradients;
    returns the final positions [V, 3] float64."""
    threads = threads or os.cpu_count() or 1
    off = np.cumsum([0] + [len(it.verts) for it in items])
    tris_g = torch.from_numpy(np.concatenate([it.tris + off[k] for k, it in enumerate(items)])).long()
    targets = []
    for it in items:
        nrm = vertex_normals_fp64(torch.from_numpy(it.verts).double(), torch.from_numpy(it.tris).long())
        r = orc.render_view(it.verts, it.tris, it.cams[0], it.H, it.W, nrm.float().numpy(), it.shading,
                            threads=threads)
        targets.append(r.image)
    verts = torch.from_numpy(np.asarray(v_init, np.float64).copy()).requires_grad_(True)
    opt = torch.optim.Adam([verts], lr=lr)
    for _ in range(steps):
        opt.zero_grad(set_to_none=True)
        nrm = vertex_normals_fp64(verts, tris_g)
        nrm_np = nrm.detach().float().numpy()
        vf = verts.detach().float().numpy()
        gv = np.zeros(verts.shape)
        gn = np.zeros(verts.shape)
        for k, it in enumerate(items):
            sl = slice(off[k], off[k + 1])
            r = orc.render_view(vf[sl], it.tris, it.cams[0], it.H, it.W, nrm_np[sl], it.shading, threads=threads)
            g = (2.0 * (r.image - targets[k])).astype(np.float32)
            gs, ga, _ = orc.backward(r.scr, r.snap, r.flags, it.tris, r.index, r.image, g, nrm_np[sl], it.shading,
                                     want_attr=True, threads=threads)
            gv[sl] += orc.project_backward(vf[sl], it.cams[0], gs)
            gn[sl] += ga
        nrm.backward(torch.from_numpy(gn))
        verts.grad += torch.from_numpy(gv)
        opt.step()
    return verts.detach().numpy()


def subset_of_batch(n_items: int = 256):
    """The four items of the uneven batch the oracle-driven loop follows: the fewest triangles, the most, and
    the items at one and two thirds of the order by triangle count."""
    from paper_2405_02508_gb300 import scenes

    nis, _ = scenes.uneven_plan(n_items)
    T = np.array([8 * n * n for n in nis])
    order = np.argsort(T, kind="stable")
    return [int(order[0]), int(order[len(order) // 3]), int(order[2 * len(order) // 3]), int(order[-1])]
