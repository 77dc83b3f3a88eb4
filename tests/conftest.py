import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built libugks.so")
    config.addinivalue_line("markers", "cpu: runs without a GPU")


def pytest_collection_modifyitems(config, items):
    import pytest
    for it in items:
        if "gpu" not in it.keywords:
            it.add_marker(pytest.mark.cpu)
