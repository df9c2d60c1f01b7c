import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libgbhegv.so")
    config.addinivalue_line("markers", "slow: long-running case")
    config.addinivalue_line("markers", "late: extended checks, run after the core parity suite")
    config.addinivalue_line("markers", "last: runs after every other test")


def pytest_collection_modifyitems(config, items):
    """Core suite first, then the tests marked late, then those marked last
    (a stable sort: the order inside each group is the collection order)."""
    def group(item):
        if item.get_closest_marker("last"):
            return 2
        return 1 if item.get_closest_marker("late") else 0
    items.sort(key=group)
