"""The C-ABI library builds, loads and exports every symbol include/mer.h declares (no GPU needed:
no compute call is made)."""
from __future__ import annotations

import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions() -> list[str]:
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(mer_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("mer_rasterize", "mer_shade", "mer_backward", "mer_edge_grad_backward", "mer_interpolate_backward",
                 "mer_project", "mer_project_backward", "mer_sync_status", "mer_workspace_size"):
        assert must in names


def test_library_loads_and_exports_every_declared_symbol():
    from paper_2405_02508_gb300 import build

    path = build.build_lib()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    from paper_2405_02508_gb300 import binding

    assert set(binding.exported_symbols()) == set(declared_functions())


def test_host_only_calls():
    """Calls that touch no device: error strings, version, workspace sizing and argument validation."""
    from paper_2405_02508_gb300 import binding

    lib = binding.lib()
    assert lib.mer_strerror(0) == b"ok"
    assert lib.mer_version() >= 1
    assert lib.mer_workspace_size(100, 200, 2, 64, 48, 16, 0) > 0
    assert lib.mer_workspace_size(100, 200, 2, 64, 48, 12, 0) == 0
    assert lib.mer_workspace_size(100, 200, 2, 9000, 48, 16, 0) == 0
    assert lib.mer_rasterize(None, 3, None, 1, 1, 16, 16, 16, None, 0, None, None, None, None, None) == binding.MER_EINVAL
    assert lib.mer_project(None, 3, None, 1, None, None) == binding.MER_EINVAL
    assert lib.mer_project(None, 0, None, 1, None, None) == binding.MER_OK  # empty: nothing to do


def test_batch_plan_offsets():
    """mer_batch_plan (host only): running offsets per item and totals; oversized items are refused."""
    from paper_2405_02508_gb300 import binding

    arr = (binding.MerItem * 3)()
    sizes = [(10, 7, 40, 50), (0, 0, 0, 0), (5, 3, 17, 33)]
    for k, (V, T, H, W) in enumerate(sizes):
        arr[k].V, arr[k].T, arr[k].H, arr[k].W = V, T, H, W
    tot = binding.mer_batch_plan(arr, 32)
    assert [arr[k].vrec for k in range(3)] == [0, 10, 10]
    assert [arr[k].trec for k in range(3)] == [0, 7, 7]
    assert [arr[k].pix for k in range(3)] == [0, 2000, 2000]
    assert [arr[k].tile for k in range(3)] == [0, 4, 4]  # ceil(50/32) * ceil(40/32) = 4
    assert [arr[k].btile for k in range(3)] == [0, 6, 6]  # backward tiles of 32 x 16: ceil(50/32) * ceil(40/16)
    assert (tot.vrecs, tot.trecs, tot.pixels, tot.tiles, tot.btiles) == (15, 10, 2000 + 561, 4 + 2, 6 + 4)
    assert binding.mer_batch_workspace_size(tot) > 0
    assert tot.mesh_rows == 10  # every item starts at world row 0 here: the largest V
    assert tot.max_tri_density == max(7 / 2000, 3 / 561)
    arr[0].H = 9000
    import pytest

    with pytest.raises(binding.MerError):
        binding.mer_batch_plan(arr, 32)


def test_backward_workspace_sizes():
    """Host-only sizing of the backward workspace: the status header alone, or with MER_DETERMINISTIC the
    fixed-point sums of the vertex and attribute gradients (each part rounded up to 256 bytes)."""
    from paper_2405_02508_gb300 import binding as B

    assert B.mer_backward_workspace_size(1000, 500, 2, 7) == 256
    det = 7 | B.MER_DETERMINISTIC
    assert B.mer_backward_workspace_size(1000, 500, 2, det) == 256 + 48128 + 16128
    assert B.mer_backward_workspace_size(10, 0, 0, det) == 256 + 512
    assert B.mer_backward_workspace_size(-1, 0, 0, det) == 0
