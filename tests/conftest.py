import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    oracle.lib()
    return oracle


@pytest.fixture(scope="session")
def mlswe_lib():
    import paper_1803_01450_gb300 as pkg
    pkg.build()
    return pkg


def rel_err(a, b):
    """Per-field max |a - b| relative to the field's max |b| (floor 1e-300)."""
    import numpy as np
    a = np.asarray(a); b = np.asarray(b)
    ax = tuple(range(1, a.ndim))
    den = np.maximum(np.abs(b).max(axis=ax), 1e-300)
    return (np.abs(a - b).max(axis=ax) / den)
