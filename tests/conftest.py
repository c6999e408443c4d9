import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _ensure_library():
    """Build libadaptive_region.so in-tree if it is missing or stale (nvcc
    cross-compiles for sm_103a without a GPU); the package refuses to import
    without it."""
    spec = importlib.util.spec_from_file_location("_ar_build", os.path.join(ROOT, "paper_2303_08873_b300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running case")
    _ensure_library()
