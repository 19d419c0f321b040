import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")


import pytest


def _gpu_visible() -> bool:
    return os.path.exists("/dev/nvidia0") or bool(os.environ.get("CUDA_VISIBLE_DEVICES"))


def pytest_collection_modifyitems(config, items):
    # GPU tests are skipped only on machines with no NVIDIA device at all; where
    # a device exists, a CUDA failure is a test failure.
    if _gpu_visible():
        return
    skip = pytest.mark.skip(reason="no NVIDIA GPU on this machine")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


@pytest.fixture(scope="session")
def evd():
    """The Python binding with libevd built in-tree (compiles on first use)."""
    from paper_2504_07059_gb300 import build, evd as binding
    build.build()
    binding.lib()
    return binding
