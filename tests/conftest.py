import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a kernels through the C ABI)")
    config.addinivalue_line("markers", "slow: long-running full-size case")


def golden_path(name: str) -> str:
    return os.path.join(ROOT, "tests", "golden", name)


@pytest.fixture(scope="session")
def orc():
    import oracle
    return oracle.load()


def pytest_sessionstart(session):
    # Build the C generators, the oracle and the CUDA library if they are missing
    # (nvcc cross-compiles without a GPU).
    lib = os.path.join(ROOT, "paper_2502_19284_gb300", "_build", "libspmv.so")
    if not os.path.exists(lib):
        import __graft_entry__
        __graft_entry__.build()


def cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False
