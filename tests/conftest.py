import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


def _cuda_ok():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def gpu():
    """Builds libsdtw.so (sm_103a) and returns torch's cuda:0; skips without a GPU."""
    if not _cuda_ok():
        pytest.skip("no CUDA device")
    import torch
    from paper_2403_06931_gb300 import build, capi
    build.build()
    capi.load()
    torch.cuda.set_device(0)
    return torch.device("cuda:0")
