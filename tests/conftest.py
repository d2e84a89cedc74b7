import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


def pytest_collection_modifyitems(config, items):
    # The test that checks the non-allocating entry point is collected last, whatever the file order.
    last = [it for it in items if os.path.basename(str(it.fspath)).startswith("test_zz_")]
    rest = [it for it in items if it not in last]
    items[:] = rest + last
