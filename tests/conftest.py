import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built extension")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def cs_gpu():
    """The product binding, with the CUDA library loaded.  A GPU test that
    cannot load it fails (it never falls back to anything)."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected but CUDA is not available")
    import paper_2501_11592_gb300 as cs
    cs.load()          # raises if the shared library is missing
    return cs
