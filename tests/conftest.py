import os
import sys
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parent.parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))
GOLDEN = Path(__file__).resolve().parent / "golden"


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and libhemegb")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def load_d3q19():
    """(c[19,3] int, w[19] float) from the golden fixture (paper Section 2.2)."""
    rows = np.loadtxt(GOLDEN / "d3q19.txt", dtype=np.int64)
    assert rows.shape == (19, 6)
    assert (rows[:, 0] == np.arange(19)).all()
    return rows[:, 1:4], rows[:, 4] / rows[:, 5]


@pytest.fixture(scope="session")
def d3q19():
    return load_d3q19()
