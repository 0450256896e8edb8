import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes tens of seconds on the CPU")


def load_golden(name):
    """Parse a tests/golden/*.txt fixture: '# comments', 'key value' and 'S th ph v...' rows."""
    scalars, rows = {}, []
    with open(os.path.join(ROOT, "tests", "golden", name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] == "S":
                rows.append([float(v) for v in parts[1:]])
            else:
                scalars[parts[0]] = float(parts[1])
    return scalars, rows
