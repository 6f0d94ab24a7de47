import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: large inputs (full-size workloads)")


def pytest_collection_modifyitems(config, items):
    # keep the file that must run last at the end regardless of collection order
    last = [it for it in items if os.path.basename(str(it.fspath)).startswith("test_zz_")]
    rest = [it for it in items if it not in last]
    items[:] = rest + last


@pytest.fixture(scope="session")
def golden_example():
    """Parses tests/golden/partition_example.txt (hand-derived values)."""
    path = os.path.join(ROOT, "tests", "golden", "partition_example.txt")
    out = {"edge": [], "stats": [], "mode": [], "bytes": []}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            if key in out:
                out[key].append([int(v) for v in vals])
            else:
                out[key] = [int(v) for v in vals]
    return out
