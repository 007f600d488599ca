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
def cdmpt_lib():
    """The built library (built in-tree on first use if missing)."""
    import paper_1503_07037_gb300 as pkg
    from paper_1503_07037_gb300 import build as b
    if not os.path.exists(pkg.LIB_PATH):
        b.build()
    return pkg


@pytest.fixture(scope="session")
def cuda(cdmpt_lib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")
