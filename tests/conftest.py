import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libntbc")
    # build libntbc.so in-tree when it is missing (nvcc cross-compiles without a GPU)
    if not os.path.exists(os.path.join(ROOT, "paper_2407_09543_gb300", "libntbc.so")):
        import __graft_entry__

        __graft_entry__.build()


def golden(name):
    """Read a tests/golden/*.txt fixture: 'key value...' lines, '#' comments."""
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, *v = line.split()
                out[k] = v
    return out
