import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running")


@pytest.fixture(scope="session")
def libec():
    """The built C-ABI library (built in-tree if missing)."""
    from paper_2311_11740_gb300 import build as _build
    _build.build()
    from paper_2311_11740_gb300 import ec
    return ec.lib()


@pytest.fixture(scope="session")
def gpu_ctx(libec):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_11740_gb300 import ec
    return ec.default_context(0)
