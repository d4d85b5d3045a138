import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def load_decompositions():
    """Parse tests/golden/decompositions.txt -> {(variant, name): np.ndarray}."""
    import numpy as np

    out, cur, rows = {}, None, []
    with open(os.path.join(GOLDEN, "decompositions.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("=="):
                if cur is not None:
                    out[cur] = np.array(rows, dtype=np.uint8)
                parts = line[2:].split()
                cur, rows = (parts[0], parts[1]), []
                continue
            rows.append([int(x) for x in line.split()])
    if cur is not None:
        out[cur] = np.array(rows, dtype=np.uint8)
    return out


@pytest.fixture(scope="session")
def decomp():
    return load_decompositions()
