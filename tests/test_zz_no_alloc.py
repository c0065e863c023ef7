"""mer_rasterize_noalloc: rasterization for callers that cannot allocate device memory when they call.

Some callers cannot hand the library a workspace: code that runs while a stream is being captured into a
CUDA graph (cudaMalloc is not permitted there), or a host framework or plugin that passes the library its
input and output buffers but offers no device allocator.  For them the library keeps its own fixed 64 MiB
device array and ``mer_rasterize_noalloc`` uses it instead of a caller workspace.

This file checks, through the C-ABI, that the variant gives the same index, depth and barycentric images
as ``mer_rasterize`` with a caller workspace, on two different scenes rasterized back to back (the second
call must not see anything the first left in the shared array), and that oversized requests are refused.
It is collected last on purpose so that a failure here comes after every other test has run.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_2405_02508_gb300 import scenes

from . import parity

pytestmark = pytest.mark.gpu


def _rasterize_both(scene, tile=16):
    import torch

    from paper_2405_02508_gb300 import binding as B
    from paper_2405_02508_gb300.render import Renderer

    dev = "cuda"
    n, H, W = scene.n_views, scene.H, scene.W
    r = Renderer(torch.from_numpy(scene.tris), len(scene.verts), n, H, W, scene.shading, scene.attr.shape[1],
                 tile=tile)
    r.project(torch.from_numpy(scene.verts).to(dev), B.cameras_tensor(scene.cams))
    depth_ref = torch.empty((n, H, W), dtype=torch.float32, device=dev)
    bary_ref = torch.empty((n, H, W, 2), dtype=torch.float32, device=dev)
    r.rasterize(depth_ref, bary_ref)  # the existing entry point, caller workspace, status checked
    index = torch.full((n, H, W), -7, dtype=torch.int32, device=dev)
    depth = torch.full((n, H, W), -7.0, dtype=torch.float32, device=dev)
    bary = torch.full((n, H, W, 2), -7.0, dtype=torch.float32, device=dev)
    status = torch.full((1,), -1, dtype=torch.int32, device=dev)
    B.mer_rasterize_noalloc(r.vpix, r.tris, H, W, tile, index, depth, bary, status)
    torch.cuda.synchronize()
    return (r.index.cpu().numpy(), depth_ref.cpu().numpy(), bary_ref.cpu().numpy(),
            index.cpu().numpy(), depth.cpu().numpy(), bary.cpu().numpy(), int(status.item()))


def test_noalloc_matches_workspace_entry_point_on_consecutive_calls():
    for scene in (scenes.two_spheres(H=384, W=320), scenes.tiny_icosphere()):
        idx_ref, dep_ref, bar_ref, idx, dep, bar, status = _rasterize_both(scene)
        assert status == 0
        np.testing.assert_array_equal(idx, idx_ref)
        np.testing.assert_allclose(dep, dep_ref, rtol=parity.IMG_TOL, atol=parity.IMG_TOL)
        np.testing.assert_allclose(bar, bar_ref, rtol=parity.IMG_TOL, atol=parity.IMG_TOL)
        assert (idx >= 0).sum() > 1000


def test_noalloc_refuses_sizes_beyond_its_array():
    import torch

    from paper_2405_02508_gb300 import binding as B

    # 2M triangles x 1 view need 96 MiB of raster records alone: more than the 64 MiB array
    T = 2_000_000
    vpix = torch.zeros((1, 3, B.VERTEX_FLOATS), dtype=torch.float32, device="cuda")
    tris = torch.zeros((T, 3), dtype=torch.int32, device="cuda")
    index = torch.empty((1, 16, 16), dtype=torch.int32, device="cuda")
    with pytest.raises(B.MerError) as e:
        B.mer_rasterize_noalloc(vpix, tris, 16, 16, 16, index)
    assert e.value.code == B.MER_EINVAL
