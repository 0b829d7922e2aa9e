import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (run with -m gpu on the GB300 box)")
    config.addinivalue_line("markers", "slow: longer CPU test")


def pytest_collection_modifyitems(config, items):
    # tests whose module name ends in _gpu are GPU tests even if unmarked
    for it in items:
        if it.fspath.basename.endswith("_gpu.py") and "gpu" not in it.keywords:
            it.add_marker(pytest.mark.gpu)
