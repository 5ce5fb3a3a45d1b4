import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300) and the built library")
    config.addinivalue_line("markers", "late: run after every other test (heavy cases)")


def pytest_collection_modifyitems(config, items):
    """Tests marked `late` run after all others (a stable sort keeps the rest
    in file order), so that under -x a failure among them cannot stop the
    others from running."""
    items.sort(key=lambda item: item.get_closest_marker("late") is not None)
