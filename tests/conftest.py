import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 GPU and the built CUDA library")


@pytest.fixture(scope="session")
def root():
    return ROOT


def _has_gpu():
    import ctypes
    try:
        rt = ctypes.CDLL("libcudart.so")
    except OSError:
        return False
    cnt = ctypes.c_int(0)
    return rt.cudaGetDeviceCount(ctypes.byref(cnt)) == 0 and cnt.value > 0


def pytest_collection_modifyitems(config, items):
    if any("gpu" in it.keywords for it in items) and not _has_gpu():
        skip = pytest.mark.skip(reason="no CUDA device")
        for it in items:
            if "gpu" in it.keywords:
                it.add_marker(skip)


@pytest.fixture(scope="session")
def gw():
    """The binding with a freshly built library (fails loudly if the build fails)."""
    from paper_1210_7683_gb300 import build as gbuild
    gbuild.build()
    import paper_1210_7683_gb300 as g
    return g


@pytest.fixture(scope="session")
def gw_cpu():
    """The binding with the library built, for host-only entry points (no GPU needed)."""
    from paper_1210_7683_gb300 import build as gbuild
    gbuild.build()
    import paper_1210_7683_gb300 as g
    return g
