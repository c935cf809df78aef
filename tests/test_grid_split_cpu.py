"""The library's grid split of coordinates (split_grid, used by every
double-float pair kernel) against its definition h = G rint(x / G),
l = g rint((x - h) / g) with g = G 2^-24 and ties to even: the device header
is compiled for the host with nvcc and checked bit for bit on random values,
exact ties on both grids, values far below the grid, zero and subnormals.
Runs on the CPU; skipped where nvcc is absent."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    return None


def test_grid_split_matches_its_definition(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "grid_split_check")
    src = os.path.join(ROOT, "tests", "grid_split_check.cu")
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-o", exe, src], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    print(r.stdout)
    assert r.returncode == 0, r.stdout[-2000:]
