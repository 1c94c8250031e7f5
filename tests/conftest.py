import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)

GOLDEN = os.path.join(HERE, "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a kernels)")
    config.addinivalue_line("markers", "slow: long-running oracle case")


@pytest.fixture(scope="session")
def golden_dir():
    return GOLDEN


def pytest_runtest_setup(item):
    if item.get_closest_marker("gpu") is not None:
        import torch

        if not torch.cuda.is_available():
            pytest.fail("GPU test selected but no CUDA device is visible", pytrace=False)


@pytest.fixture(scope="session")
def nsg():
    """The CUDA library, built in-tree for sm_103a (fails loudly if it cannot be)."""
    from paper_1707_00143_gb300 import build, capi

    build.build()
    capi.lib()
    return capi
