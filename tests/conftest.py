import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: full-size parity cases (minutes)")


def load_worked_example():
    """Parse tests/golden/worked_example.txt into a dict."""
    path = os.path.join(ROOT, "tests", "golden", "worked_example.txt")
    out = {"nnz": [], "prefix": [], "segment": []}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *rest = line.split()
            vals = [int(x) for x in rest]
            if key in ("nnz", "prefix", "segment"):
                out[key].append(vals)
            elif key == "dims":
                out[key] = vals
            else:
                out[key] = vals[0]
    return out


@pytest.fixture
def worked_example():
    return load_worked_example()
