import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# The ragged batcher's tuning table persists in a file by default; tests that
# count tuning runs must not see choices an earlier process left there, so the
# session runs without one unless the caller names a file
# (tests/test_alloc_and_tuning.py gives its child processes their own).
os.environ.setdefault("ORAND_TUNE_CACHE", "off")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    return oracle
