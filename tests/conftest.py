import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300); runs the CUDA path through the C ABI")
    config.addinivalue_line("markers", "slow: full-size workloads")


@pytest.fixture(scope="session")
def ctx():
    """One grid context on cuda:0 for the GPU tests."""
    import paper_2403_10647_gb300 as pg
    from paper_2403_10647_gb300 import build as pbuild
    pbuild.build_library()
    c = pg.Context(0)
    yield c
    c.close()
