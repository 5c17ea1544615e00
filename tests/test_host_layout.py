"""Host check of the single-dataset workspace layout, linked against the built
library: aligned, non-overlapping regions, each large enough for what reads or
writes it (including the split partials of every order's plan and the kept
order-4 moments), over a grid of sizes, orders, block sides and precisions."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host", "layout_check.cu")
LIBDIR = os.path.join(ROOT, "paper_1701_05420_gb300", "_lib")
EXE = os.path.join(ROOT, "_build", "tests", "layout_check")


def test_workspace_layout():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    assert os.path.exists(os.path.join(LIBDIR, "libcumgb.so")), "build the library first"
    os.makedirs(os.path.dirname(EXE), exist_ok=True)
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "--expt-relaxed-constexpr",
                        "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_1701_05420_gb300", "csrc"),
                        SRC, "-o", EXE, "-L", LIBDIR, "-lcumgb", "-Xlinker", "-rpath", "-Xlinker", LIBDIR],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([EXE], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "0 failures" in r.stdout
