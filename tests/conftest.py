import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _ensure_built():
    """Build libcumgb.so in-tree if it is missing (nvcc cross-compiles without a GPU)."""
    lib = os.path.join(ROOT, "paper_1701_05420_gb300", "_lib", "libcumgb.so")
    if os.path.exists(lib):
        return
    spec = importlib.util.spec_from_file_location("_cumgb_build", os.path.join(ROOT, "paper_1701_05420_gb300",
                                                                               "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    _ensure_built()
