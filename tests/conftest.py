import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden_dfa(name):
    """Parse a figure fixture: returns (n, k, start or None, accepting names, edges, names)."""
    import numpy as np
    header = {}
    edges = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] in ("states", "letters", "start", "accepting"):
                header[parts[0]] = parts[1:]
            else:
                edges.append((parts[0], int(parts[1]), parts[2]))
    return header, edges
