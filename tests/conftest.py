"""Shared pytest set-up: the gpu marker and the repository root on sys.path."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libsw")
    config.addinivalue_line("markers", "slow: long CPU-only statistical check")


def build_libsw():
    """Build libsw.so (if stale) without importing the package, whose import
    loads the library and raises while it is missing."""
    import importlib.util
    path = os.path.join(ROOT, "paper_2302_14720_gb300", "build.py")
    spec = importlib.util.spec_from_file_location("_libsw_build", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build()
