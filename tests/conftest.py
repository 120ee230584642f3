import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def tiny_inputs():
    """The plain-method tiny workload: 4 depth maps 320x96 and their poses."""
    from synth.scenes import tiny_scene
    s = tiny_scene(seed=0)
    return s, s.depth_maps()
