import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def nsdf_lib():
    """The built C-ABI library (compiled in-tree for sm_103a if stale)."""
    from paper_2110_01614_gb300 import build
    build.ensure_built()
    import paper_2110_01614_gb300 as nsdf
    return nsdf.library()
