"""Pins of the Laplacian-preconditioning oracle (Nicolet et al.'s large-steps reparameterisation, used by the
paper for every mesh optimisation) against mathematics that is not the oracle itself: known graph spectra,
brute-force neighbour counts, the constant null space, exact round trips."""
from __future__ import annotations

import itertools

import numpy as np
import pytest

from paper_2405_02508_gb300 import scenes


@pytest.fixture(scope="module")
def lap():
    from oracle import laplacian

    return laplacian


def _brute_neighbours(tris, V):
    nb = [set() for _ in range(V)]
    for t in tris:
        for a, b in itertools.permutations([int(v) for v in t], 2):
            if a != b:
                nb[a].add(b)
    return nb


def test_icosahedron_spectrum(lap):
    """The icosahedron's graph Laplacian has eigenvalues 0, 5 - sqrt5 (x3), 6 (x5), 5 + sqrt5 (x3)."""
    P, F = scenes.icosphere(0)
    assert len(P) == 12 and len(F) == 20
    ev = np.sort(np.linalg.eigvalsh(lap.laplacian(F, 12).toarray()))
    s5 = np.sqrt(5.0)
    expect = np.sort([0.0] + [5 - s5] * 3 + [6.0] * 5 + [5 + s5] * 3)
    np.testing.assert_allclose(ev, expect, atol=1e-12)


def test_tetrahedron_spectrum_and_system(lap):
    """K4: L = 4I - J, eigenvalues 0, 4, 4, 4; so M = I + lam L has 1, 1 + 4 lam (x3)."""
    F = np.array([[0, 1, 2], [0, 3, 1], [1, 3, 2], [2, 3, 0]])
    L = lap.laplacian(F, 4).toarray()
    np.testing.assert_array_equal(L, 4 * np.eye(4) - np.ones((4, 4)))
    ev = np.sort(np.linalg.eigvalsh(lap.system(F, 4, 16.0).toarray()))
    np.testing.assert_allclose(ev, [1.0, 65.0, 65.0, 65.0], rtol=1e-14)


@pytest.mark.parametrize("mesh", ["octasphere", "open_sphere", "degenerate"])
def test_degrees_symmetry_and_null_space(lap, mesh):
    """Diagonal = brute-force neighbour counts, off-diagonal -1 exactly on neighbours, symmetric, rows sum to
    zero (constants in the null space), for closed, open and degenerate-edge meshes."""
    if mesh == "octasphere":
        P, F = scenes.octasphere(4)
    elif mesh == "open_sphere":
        sc = scenes.open_sphere(H=16, W=16, subdiv=2)
        P, F = sc.verts, sc.tris
    else:
        P, F = scenes.icosphere(1)
        F = np.concatenate([F, [[0, 0, 5], [3, 7, 3]]])
    V = len(P)
    L = lap.laplacian(F, V).toarray()
    nb = _brute_neighbours(F, V)
    for i in range(V):
        assert L[i, i] == len(nb[i])
        row = L[i].copy()
        row[i] = 0
        assert set(np.nonzero(row)[0]) == nb[i]
        assert np.all(row[list(nb[i])] == -1.0)
    np.testing.assert_array_equal(L, L.T)
    np.testing.assert_array_equal(L.sum(axis=1), 0.0)


def test_solve_round_trip_constants_and_eigenvectors(lap):
    """M^-1 (M x) = x; a constant field is unchanged by M^-1 (translation passes through the preconditioner
    untouched); and M^-1 scales every eigenvector v of L (dense symmetric eigensolver) by 1 / (1 + lam mu), so
    rough fields are damped far more than smooth ones."""
    P, F = scenes.octasphere(6)
    V = len(P)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((V, 3))
    np.testing.assert_allclose(lap.solve(F, V, 16.0, lap.apply(F, V, 16.0, x)), x, rtol=0, atol=1e-10)
    c = np.tile([[0.3, -1.2, 2.5]], (V, 1))
    np.testing.assert_allclose(lap.solve(F, V, 16.0, c), c, rtol=0, atol=1e-12)
    mu, vec = np.linalg.eigh(lap.laplacian(F, V).toarray())
    pick = [1, 5, V // 2, V - 1]
    b = np.stack([vec[:, k] for k in pick[:3]], axis=1)
    np.testing.assert_allclose(lap.solve(F, V, 16.0, b), b / (1.0 + 16.0 * mu[pick[:3]]), atol=1e-12)
    top = lap.solve(F, V, 16.0, np.repeat(vec[:, [V - 1]], 3, axis=1))[:, 0]
    assert np.linalg.norm(top) == pytest.approx(1.0 / (1.0 + 16.0 * mu[V - 1]), rel=1e-10)
    assert 1.0 / (1.0 + 16.0 * mu[V - 1]) < 0.01


def test_uniform_adam_reduces_to_sign_steps_on_first_step(lap):
    """First step of Adam: m_hat = g, v_hat = g^2, so each block moves by lr * g / max|g| (eps aside);
    two blocks use their own maxima."""
    g = np.array([[1.0, -2.0, 0.5], [4.0, 0.0, -1.0], [0.1, 0.2, -0.3]])
    opt = lap.UniformAdam(g.shape, [(0, 2), (2, 3)], lr=0.1, eps=0.0)
    out = opt.step(np.zeros_like(g), g)
    np.testing.assert_allclose(out[:2], -0.1 * g[:2] / 4.0, rtol=1e-14)
    np.testing.assert_allclose(out[2:], -0.1 * g[2:] / 0.3, rtol=1e-14)
