import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libgvt")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


def read_golden_matrices(name):
    """Parse a tests/golden text fixture made of '[NAME rows cols]' blocks."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", name)
    out, cur, rows = {}, None, []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                if cur:
                    out[cur] = np.array(rows, dtype=float)
                cur, rows = line[1:-1].split()[0], []
            else:
                rows.append([float(x) for x in line.split()])
    if cur:
        out[cur] = np.array(rows, dtype=float)
    return out
