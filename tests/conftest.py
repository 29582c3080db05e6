import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libtgf")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def tgf():
    """The CUDA library binding; GPU tests only."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_03747_gb300 import build

    build.build()
    from paper_2107_03747_gb300 import binding

    return binding
