import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: full-size parity case")


class SimpleView:
    """A camera given directly by its row-major view-projection matrix."""

    def __init__(self, m, width, height, znear, zfar):
        import numpy as np
        self.viewproj = np.ascontiguousarray(np.asarray(m, np.float32).reshape(16))
        self.width, self.height, self.znear, self.zfar = width, height, znear, zfar


@pytest.fixture
def simple_view():
    return SimpleView
