import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def golden(name):
    """Parse tests/golden/paper_values.txt -> value (int, float or tuple)."""
    path = os.path.join(ROOT, "tests", "golden", "paper_values.txt")
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = (s.strip() for s in line.split("=", 1))
            if k == name:
                if "," in v:
                    return tuple(float(x) for x in v.split(","))
                return int(v) if v.lstrip("-").isdigit() else float(v)
    raise KeyError(name)


@pytest.fixture
def gold():
    return golden
