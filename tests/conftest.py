import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line(
        "markers", "slow: oracle work of tens of seconds")


def pytest_collection_modifyitems(config, items):
    # keep a run that stops at the first failure informative: files whose
    # name sorts last run last
    items.sort(key=lambda it: os.path.basename(str(it.fspath)))
