import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU-only test (minutes)")


def pytest_collection_modifyitems(config, items):
    # tests marked slow run only when asked for explicitly (-m slow)
    mexpr = config.getoption("-m") or ""
    if "slow" in mexpr:
        return
    skip = pytest.mark.skip(reason="slow CPU test; run with -m slow")
    for it in items:
        if "slow" in it.keywords:
            it.add_marker(skip)
