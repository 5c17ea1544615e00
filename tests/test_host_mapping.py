"""Host check of the staircase contraction's index mapping, compiled from the
library's own header (csrc/common.cuh) with nvcc as host code: every valid
(row, column) pair of the Khatri-Rao GEMM lands on the block-storage address
of its entry (colex rank of the sorted block tuple, C order inside the block),
every stored entry is produced exactly once, and the tile staircase covers
every tile that holds a valid pair."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host", "mapping_check.cu")
CSRC = os.path.join(ROOT, "paper_1701_05420_gb300", "csrc")
EXE = os.path.join(ROOT, "_build", "tests", "mapping_check")


@pytest.fixture(scope="module")
def exe():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    os.makedirs(os.path.dirname(EXE), exist_ok=True)
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-I", CSRC, SRC, "-o", EXE], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return EXE


@pytest.mark.parametrize("d,n,b", [
    (2, 7, 3), (3, 10, 2), (4, 9, 2), (4, 20, 4), (5, 10, 2), (5, 13, 3), (6, 8, 2), (6, 12, 2),
    (3, 48, 16), (4, 1, 1), (6, 3, 4), (2, 64, 64),
])
@pytest.mark.parametrize("tile", [128, 256])
def test_mapping_is_a_bijection_onto_block_storage(exe, d, n, b, tile):
    r = subprocess.run([exe, str(d), str(n), str(b), str(tile)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
