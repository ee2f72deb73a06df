"""The lattice index arithmetic of the CUDA kernels (site coordinates by
multiply-shift division, neighbour half indices by additive offsets), compiled
from the kernels' own header for the host and checked on the CPU against plain
division and periodic coordinate arithmetic on ten lattices, including
extents of 2 and unequal extents."""
import os
import subprocess

import pytest

from paper_0904_1179_gb300 import build as su3_build

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_index_arithmetic_on_host(tmp_path):
    try:
        nvcc = su3_build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "index_host")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O2",
                    "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_0904_1179_gb300", "csrc"),
                    "-o", exe, os.path.join(HERE, "index_host.cu")], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-3000:]
    assert "index arithmetic ok" in r.stdout
