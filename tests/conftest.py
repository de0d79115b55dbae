import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


@pytest.fixture(scope="session")
def hull_lib():
    """The CUDA library through its C ABI (builds it if it is missing)."""
    from paper_1508_05931_gb300 import build as _b
    _b.build_library()
    from paper_1508_05931_gb300 import hull
    return hull
