import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def capi():
    """The CUDA C-ABI library, built in-tree (nvcc cross-compiles without a GPU)."""
    from paper_0712_0813_gb300 import build as pkg_build
    pkg_build.build()
    from paper_0712_0813_gb300 import capi as _capi
    return _capi


@pytest.fixture(scope="session")
def gpu_capi(capi):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected without a CUDA device")
    return capi
