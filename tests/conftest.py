import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built C-ABI library")
    config.addinivalue_line("markers", "slow: long-running CPU oracle case")

# GPU tests run the library with host-side bounds validation of every launch
os.environ.setdefault("IFMM_VALIDATE", "1")
