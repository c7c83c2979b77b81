import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU check")


@pytest.fixture(scope="session")
def qs():
    """The CUDA library's Python binding, built for sm_103a if needed.

    GPU tests fail (they do not skip) when no GPU or no library is present,
    so a missing build can never pass silently."""
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2008_00216_gb300 as pkg
    pkg.load()                       # raises if the shared library is missing
    return pkg
