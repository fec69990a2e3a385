import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


def dense_from_csc(n, colptr, rowidx, values=None):
    M = np.zeros((n, n))
    for j in range(n):
        for p in range(colptr[j], colptr[j + 1]):
            M[rowidx[p], j] = 1.0 if values is None else values[p]
    return M


def csc_from_mask(mask):
    n = mask.shape[0]
    colptr = np.zeros(n + 1, np.int64)
    rows = []
    for j in range(n):
        r = np.nonzero(mask[:, j])[0]
        rows.append(r)
        colptr[j + 1] = colptr[j] + r.size
    return colptr, (np.concatenate(rows) if rows else np.zeros(0)).astype(np.int32)


@pytest.fixture(scope="session")
def grid32():
    import synth
    return synth.make("grid32_natural", 0)
