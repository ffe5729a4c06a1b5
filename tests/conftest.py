import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def oracle():
    import oracle as o
    o.lib()
    return o


@pytest.fixture(scope="session")
def fszlib():
    """The CUDA library, built in-tree for sm_103a (no CPU fallback exists)."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_2607_15413_gb300 import fsz
    return fsz
