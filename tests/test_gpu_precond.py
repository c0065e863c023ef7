"""Laplacian preconditioning on the device (conjugate-gradient solves of I + lambda L) against the FP64
oracle's sparse direct solve, and the preconditioned uneven-batch fit against the same loop driven by the
oracle."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2405_02508_gb300 import scenes

pytestmark = pytest.mark.gpu


def _batch_mesh(n_items=4, t_max=20000):
    its = scenes.uneven_batch(n_items=n_items, t_max=t_max, resolutions=(64,))
    off = np.cumsum([0] + [len(it.verts) for it in its])
    P = np.concatenate([it.verts for it in its]).astype(np.float64)
    F = np.concatenate([it.tris + off[k] for k, it in enumerate(its)]).astype(np.int32)
    return P, F


@pytest.mark.parametrize("lam", [8.0, 16.0, 32.0])
def test_apply_and_solve_match_oracle(lam):
    from oracle import laplacian as lap

    from paper_2405_02508_gb300.precond import LaplacianPreconditioner

    P, F = _batch_mesh()
    V = len(P)
    pc = LaplacianPreconditioner(F, V, lam, max_iters=400, rel_tol=1e-7)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((V, 3)).astype(np.float32)
    y = pc.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = lap.apply(F, V, lam, x.astype(np.float64))
    np.testing.assert_allclose(y, ref, rtol=1e-5, atol=1e-5 * np.abs(ref).max())
    for b in (x, P.astype(np.float32) + 0.01 * x):  # a rough and a smooth right-hand side
        sol = pc.solve(torch.from_numpy(b).cuda()).cpu().numpy()
        it, res = pc.last_solve()
        exact = lap.solve(F, V, lam, b.astype(np.float64))
        assert res <= 1e-6 and 0 < it < 400
        np.testing.assert_allclose(sol, exact, rtol=0, atol=2e-5 * np.abs(exact).max())


def test_solve_warm_start_and_constants():
    """From the exact solution the solve does no iteration; a constant field solves to itself."""
    from oracle import laplacian as lap

    from paper_2405_02508_gb300.precond import LaplacianPreconditioner

    P, F = _batch_mesh(n_items=2, t_max=5000)
    V = len(P)
    pc = LaplacianPreconditioner(F, V, 16.0, rel_tol=1e-5)
    b = torch.from_numpy(np.random.default_rng(4).standard_normal((V, 3)).astype(np.float32)).cuda()
    exact = torch.from_numpy(lap.solve(F, V, 16.0, b.cpu().numpy().astype(np.float64)).astype(np.float32)).cuda()
    pc.solve(b, exact)
    assert pc.last_solve()[0] == 0
    c = torch.tensor([[0.5, -1.0, 2.0]], device="cuda").repeat(V, 1)
    np.testing.assert_allclose(pc.solve(c).cpu().numpy(), c.cpu().numpy(), atol=1e-5)


def oracle_precond_fit(items, v_init: np.ndarray, steps: int, lr: float, lam: float) -> np.ndarray:
    """The large-steps loop with FP64 oracle gradients and direct solves (test infrastructure)."""
    import oracle
    from oracle import laplacian as lap

    from paper_2405_02508_gb300.fit import vertex_normals

    off = np.cumsum([0] + [len(it.verts) for it in items])
    F = np.concatenate([it.tris + off[k] for k, it in enumerate(items)]).astype(np.int32)
    V = off[-1]
    tris_g = torch.from_numpy(F).long()
    targets = []
    for it in items:
        nrm = vertex_normals(torch.from_numpy(it.verts).double(), torch.from_numpy(it.tris).long()).float().numpy()
        targets.append(oracle.render_view(it.verts, it.tris, it.cams[0], it.H, it.W, nrm, it.shading).image)
    x = v_init.astype(np.float64)
    u = lap.apply(F, V, lam, x)
    opt = lap.UniformAdam(x.shape, [(off[k], off[k + 1]) for k in range(len(items))], lr)
    for _ in range(steps):
        xt = torch.from_numpy(x).requires_grad_(True)
        nrm = vertex_normals(xt, tris_g)
        nrm_np = nrm.detach().float().numpy()
        vf = x.astype(np.float32)
        gv = np.zeros_like(x)
        gn = np.zeros_like(x)
        for k, it in enumerate(items):
            sl = slice(off[k], off[k + 1])
            r = oracle.render_view(vf[sl], it.tris, it.cams[0], it.H, it.W, nrm_np[sl], it.shading)
            g = (2.0 * (r.image - targets[k])).astype(np.float32)
            gs, ga, _ = oracle.backward(r.scr, r.snap, r.flags, it.tris, r.index, r.image, g, nrm_np[sl], it.shading,
                                        want_attr=True)
            gv[sl] += oracle.project_backward(vf[sl], it.cams[0], gs)
            gn[sl] += ga
        nrm.backward(torch.from_numpy(gn))
        gx = gv + xt.grad.numpy()
        u = opt.step(u, lap.solve(F, V, lam, gx))
        x = lap.solve(F, V, lam, u)
    return x


def test_preconditioned_fit_tracks_oracle_and_converges():
    from paper_2405_02508_gb300.fit import UnevenFit

    items = scenes.uneven_batch(n_items=4, seed=21, t_min=500.0, t_max=3000.0, resolutions=(128, 192))
    fit = UnevenFit(items, sigma=0.01, seed=11)
    steps, lr, lam = 40, 2e-3, 16.0
    v_gpu = fit.run_preconditioned(steps, lr=lr, lam=lam)
    r0, r_gpu = fit.rmse(fit.v_init), fit.rmse(v_gpu)
    l0, l_gpu = fit.loss(fit.v_init), fit.loss(v_gpu)
    v_orc = oracle_precond_fit(items, fit.v_init.cpu().numpy(), steps, lr, lam)
    r_orc = fit.rmse(torch.from_numpy(v_orc.astype(np.float32)).cuda())
    print(f"rmse {r0:.5f} -> gpu {r_gpu:.5f} / oracle-driven {r_orc:.5f}; loss {l0:.1f} -> {l_gpu:.1f}")
    assert l_gpu < l0
    assert abs(r_gpu - r_orc) <= 0.02 * r_orc, (r0, r_gpu, r_orc)
