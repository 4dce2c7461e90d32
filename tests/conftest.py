import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# a cycle graph that fails to capture is an error in the tests, not a
# silent switch to host-issued cycles (tests that want those set
# SIF_NO_GRAPH=1 for their contexts)
os.environ.setdefault("SIF_REQUIRE_GRAPHS", "1")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on one CPU core")
