"""mer_laplacian_csr (a host call of the library, no GPU): the CSR edge graph equals the oracle's edge set on
closed, open and degenerate meshes and on a batch of several meshes; bad ids are refused."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from paper_2405_02508_gb300 import scenes


def _oracle_neighbours(F, V):
    from oracle import laplacian as lap

    nb = [[] for _ in range(V)]
    for a, b in lap.edge_pairs(F):
        nb[a].append(int(b))
        nb[b].append(int(a))
    return [sorted(x) for x in nb]


@pytest.mark.parametrize("mesh", ["octasphere", "open_sphere", "degenerate", "batch"])
def test_csr_equals_oracle_edge_graph(mesh):
    from paper_2405_02508_gb300 import binding as B

    if mesh == "octasphere":
        P, F = scenes.octasphere(7)
    elif mesh == "open_sphere":
        sc = scenes.open_sphere(H=16, W=16, subdiv=3)
        P, F = sc.verts, sc.tris
    elif mesh == "degenerate":
        P, F = scenes.icosphere(2)
        F = np.concatenate([F, [[0, 0, 5], [3, 7, 3], [9, 9, 9]]]).astype(np.int32)
    else:
        its = scenes.uneven_batch(n_items=3, t_max=3000, resolutions=(64,))
        off = np.cumsum([0] + [len(it.verts) for it in its])
        P = np.concatenate([it.verts for it in its])
        F = np.concatenate([it.tris + off[k] for k, it in enumerate(its)]).astype(np.int32)
    V = len(P)
    row_ptr, col = B.mer_laplacian_csr(F, V)
    nb = _oracle_neighbours(F, V)
    assert row_ptr[0] == 0 and row_ptr[-1] == sum(len(x) for x in nb)
    for i in range(V):
        assert list(col[row_ptr[i]:row_ptr[i + 1]]) == nb[i]


def test_csr_refuses_out_of_range_ids():
    from paper_2405_02508_gb300 import binding as B

    F = np.array([[0, 1, 5]], np.int32)
    rp = np.zeros(4, np.int64)
    rc = B.lib().mer_laplacian_csr(F.ctypes.data_as(ctypes.c_void_p), 1, 3, rp.ctypes.data_as(ctypes.c_void_p), None)
    assert rc == B.MER_ERANGE
    assert B.lib().mer_laplacian_csr(None, 1, 3, rp.ctypes.data_as(ctypes.c_void_p), None) == B.MER_EINVAL
