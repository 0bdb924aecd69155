import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: large CPU-side case")


@pytest.fixture(scope="session")
def cell1():
    """The 8-centre diamond cell (N=32, n=16, 24^3 grid, N_aux=256), with chi."""
    from cellgen import build_cell, config_spec
    return build_cell(config_spec(1), keep_chi=True)
