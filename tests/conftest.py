import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def pytest_sessionstart(session):
    # the CUDA library and the oracle are built in-tree; build them when a
    # fresh checkout runs the tests before any build step
    from paper_1806_04960_gb300 import build as b
    from oracle import oracle
    if not os.path.exists(b.OUT):
        b.build()
    oracle.build()
