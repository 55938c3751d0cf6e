import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libmstress")
    config.addinivalue_line("markers", "slow: long-running oracle case")


def pytest_collection_modifyitems(config, items):
    # run the no-allocation entry point's test file last (it is named test_zz_*)
    items.sort(key=lambda it: 1 if "test_zz_" in it.nodeid else 0)
