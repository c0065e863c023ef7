"""rcp_nr, the reciprocal the kernels use for 1 / (twice the area) and 1 / sum(lambda zeta), against the
correctly rounded reciprocal: on every positive float from 2^-60 to 2^60 it differs in at most one unit in the
last place, and only in a small share of the inputs."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_rcp_nr_against_correct_rounding(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "rcp_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-I", os.path.join(ROOT, "include"), "-o", exe,
                    os.path.join(ROOT, "tests", "gpu_src", "rcp_check.cu")], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    diff, worst, total = (int(v) for v in r.stdout.split())
    assert worst <= 1, f"largest difference {worst} ulp"
    assert diff <= total // 100, f"{diff} of {total} inputs differ from the correctly rounded reciprocal"
