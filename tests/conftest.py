import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the compiled library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def idg_mod():
    """The ctypes binding with libidg.so built in-tree (nvcc cross-compiles
    without a GPU)."""
    from paper_2502_17789_gb300 import build as _build
    from paper_2502_17789_gb300 import idg
    _build.build()
    idg.load()
    return idg


@pytest.fixture(scope="session")
def cuda_device():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs CUDA (run with -m 'not gpu' on a CPU-only machine)")
    return torch.device("cuda:0")
