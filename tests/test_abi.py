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
    assert lib.mer_rasterize(None, 3, None, 1, 1, 16, 16, 16, None, 0, None, None, None, None) == binding.MER_EINVAL
    assert lib.mer_project(None, 3, None, 1, None, None) == binding.MER_EINVAL
    assert lib.mer_project(None, 0, None, 1, None, None) == binding.MER_OK  # empty: nothing to do
