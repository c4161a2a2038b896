"""Shared test configuration.

Markers: tests that need a GB300 are marked ``gpu``; everything else runs on
the CPU.  The repository root is put on ``sys.path`` so that the package, the
oracle (test infrastructure) and the input generators import directly.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU statistical test")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build_oracle()
    return oracle
