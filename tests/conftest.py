import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU case")


def read_table(name):
    """Read a golden table: '#' lines are comments (citations); first
    non-comment line is the header of column labels, then one row per line:
    label value value ..."""
    path = os.path.join(ROOT, "tests", "golden", name)
    rows, header = {}, None
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if header is None:
                header = parts[1:]
                continue
            rows[parts[0]] = [None if p == "-" else float(p) for p in parts[1:]]
    return header, rows
