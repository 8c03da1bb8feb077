import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built extension")
    config.addinivalue_line("markers", "slow: long-running (large synthetic scenes)")


@pytest.fixture(scope="session")
def dv():
    """The CUDA binding, built in-tree; GPU tests fail loudly if it cannot load."""
    import paper_2606_23031_gb300 as m
    m.load()
    return m


@pytest.fixture(scope="session")
def config2_scene():
    """The 1920x1080 compositional scene (500k background leaves, 3 actors), generated once."""
    import synth
    return synth.config2(0)
