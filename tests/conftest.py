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


def first_cycle_estimate_count(N, A, f, P, target, kmax=12):
    """Iteration at which the least-squares residual estimate of the first
    FGMRES cycle (MGS Arnoldi on the oracle's A, right-preconditioned with
    the oracle's P, zero initial guess) meets the target, or None."""
    import numpy as np
    import oracle
    beta = np.linalg.norm(f)
    V, H = [f / beta], np.zeros((kmax + 1, kmax))
    for j in range(kmax):
        w = oracle.apply(N, A, P.apply(V[j])[0])
        for i in range(j + 1):
            H[i, j] = w @ V[i]
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        V.append(w / H[j + 1, j])
        e1 = np.zeros(j + 2)
        e1[0] = beta
        y = np.linalg.lstsq(H[: j + 2, : j + 1], e1, rcond=None)[0]
        if np.linalg.norm(e1 - H[: j + 2, : j + 1] @ y) <= target:
            return j + 1
    return None
