import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def orc():
    from oracle import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def nbody_lib():
    """Build (if stale) and load libnbody.so."""
    from paper_1104_2700_gb300 import build, nbody
    build.build()
    nbody.load()
    return nbody


@pytest.fixture(scope="session")
def gpu(nbody_lib):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected but no CUDA device is visible")
    return nbody_lib
