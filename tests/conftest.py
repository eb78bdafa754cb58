import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_sessionstart(session):
    """A fresh checkout has no built library: compile it (nvcc for sm_103a, in tree) before the tests that load
    it.  An existing build is used as it is."""
    from paper_2107_12330_b300 import build as libbuild
    if not os.path.exists(libbuild.LIB):
        libbuild.build()


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300) and the built libtripoll.so")
    config.addinivalue_line("markers", "slow: full-size workloads (minutes)")


def _cuda_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if _cuda_available():
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)
