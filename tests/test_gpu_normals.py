"""Vertex-normal kernels (forward and backward) against PyTorch autograd of the same formula in FP64."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2405_02508_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mesh", ["octasphere", "open_sphere", "degenerate"])
def test_vertex_normals_match_autograd(mesh):
    from paper_2405_02508_gb300.fit import VertexNormals, vertex_normals

    if mesh == "octasphere":
        P, F = scenes.octasphere(24)
    elif mesh == "open_sphere":
        sc = scenes.open_sphere(H=16, W=16, subdiv=3)
        P, F = sc.verts, sc.tris
    else:  # repeated / collapsed triangles and an isolated vertex
        P, F = scenes.icosphere(2)
        P = np.concatenate([P, [[5.0, 5.0, 5.0]]])
        F = np.concatenate([F, [[0, 0, 5], [3, 7, 3], F[0]]]).astype(np.int32)
    rng = np.random.default_rng(2)
    P = (P + rng.normal(0, 0.01, P.shape)).astype(np.float32)
    v = torch.from_numpy(P).cuda().requires_grad_(True)
    t32 = torch.from_numpy(np.ascontiguousarray(F, np.int32)).cuda()
    n = VertexNormals.apply(v, t32)
    g = torch.from_numpy(rng.standard_normal(P.shape).astype(np.float32)).cuda()
    (n * g).sum().backward()
    v64 = torch.from_numpy(P).double().requires_grad_(True)
    n64 = vertex_normals(v64, torch.from_numpy(F).long())
    (n64 * g.cpu().double()).sum().backward()
    np.testing.assert_allclose(n.detach().cpu().numpy(), n64.detach().numpy(), rtol=0, atol=2e-6)
    ref = v64.grad.numpy()
    np.testing.assert_allclose(v.grad.cpu().numpy(), ref, rtol=1e-4, atol=1e-4 * np.abs(ref).max())
