import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libmdot")
    config.addinivalue_line("markers", "slow: long CPU test")
    config.addinivalue_line("markers", "timeout(seconds): per-test limit (pytest-timeout)")


def pytest_collection_modifyitems(config, items):
    # Keep files whose name starts with test_zz_ at the very end of the run.
    items.sort(key=lambda it: os.path.basename(str(it.fspath)).startswith("test_zz_"))
