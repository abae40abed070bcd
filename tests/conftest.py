import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled library")
    config.addinivalue_line("markers", "slow: large inputs (seconds of CPU work)")


@pytest.fixture(scope="session")
def gi():
    """The CUDA library binding; GPU tests only."""
    import paper_1805_00923_gb300 as gi_mod
    return gi_mod
