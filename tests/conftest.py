import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def load_hand_examples():
    """Parse tests/golden/hand_examples.txt into a list of dicts."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", "hand_examples.txt")
    lines = [ln.strip() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    out, i = [], 0
    while i < len(lines):
        name = lines[i].split()[1]
        _, n, d = lines[i + 1].split()
        n, d = int(n), int(d)
        pts = np.array([[int(v) for v in lines[i + 2 + r].split()] for r in range(n)],
                       dtype=np.int64).reshape(n, d)
        j = i + 2 + n
        z = np.array([int(v) for v in lines[j].split()[1:]], dtype=np.int64)
        l1 = np.array([int(v) for v in lines[j + 1].split()[1:]], dtype=np.int64)
        l2 = np.array([int(v) for v in lines[j + 2].split()[1:]], dtype=np.int64)
        out.append(dict(name=name, X=pts, z=z, l1=l1, l2sq=l2))
        i = j + 3
    return out
