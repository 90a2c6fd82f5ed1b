import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libsimplex")
    config.addinivalue_line("markers", "slow: full-size configuration (minutes of oracle work)")


@pytest.fixture(scope="session")
def oracle():
    import oracle as _oracle
    _oracle.build()
    return _oracle


@pytest.fixture(scope="session")
def gpu():
    """The CUDA library on a GPU; tests marked gpu use it."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_07394_gb300 import build as _build
    import paper_1610_07394_gb300 as _sx
    _build.build()
    _sx.lib()
    return _sx

