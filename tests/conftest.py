"""Shared pytest set-up: the `gpu` marker and loaders for the three
independent libraries (generators, oracle, CUDA path)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def read_golden(name):
    """Parse a `key: value` fixture under tests/golden/ (# lines are notes)."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(":", 1)
            out[k.strip()] = v.strip()
    return out


def ints(s):
    return [int(x) for x in s.split()]


@pytest.fixture(scope="session")
def orc():
    import oracle
    return oracle.get()
