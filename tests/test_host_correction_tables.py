"""Host check of the correction kernel's compile-time partition tables
(csrc/correct.cu), built with nvcc as a host program that includes the kernel
source: evaluated the way the staged kernel evaluates them (two-part products,
three-pair groups, and the order-6 moment form reading M_4), they must equal a
direct sum over independently enumerated set partitions of 1:d into >= 2 parts
of size >= 2 (Eq. cum_r), for d = 4, 5, 6."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host", "correction_tables_check.cu")
EXE = os.path.join(ROOT, "_build", "tests", "correction_tables_check")


def test_partition_tables_match_direct_sum():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    os.makedirs(os.path.dirname(EXE), exist_ok=True)
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "--expt-relaxed-constexpr",
                        "-gencode", "arch=compute_103a,code=sm_103a",
                        "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_1701_05420_gb300", "csrc"),
                        SRC, "-o", EXE], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([EXE], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "d=6 partitions=40" in r.stdout
