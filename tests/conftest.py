import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs on the GB300 box)")
    config.addinivalue_line("markers", "slow: long-running CPU case")


def pytest_collection_finish(session):
    """Modules with long oracle runs expose start_background_oracles(); start them as soon
    as one of their tests is selected, so that they overlap the rest of the session."""
    started = set()
    for item in session.items:
        mod = getattr(item, "module", None)
        start = getattr(mod, "start_background_oracles", None)
        if start is not None and mod.__name__ not in started:
            started.add(mod.__name__)
            start()
