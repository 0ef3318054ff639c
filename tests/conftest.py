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


G = 9.81


def state_scale(q_ref, M, g=G):
    """Per-field scale of the state parity bounds (fields (h, hu, hv) per layer): a depth,
    its own largest value; a momentum, the larger of its own largest magnitude and
    h_max sqrt(g h_max), the momentum of the layer's deepest column moving at its own
    gravity-wave speed. The physical floor keeps the bound meaningful where the flow is
    near rest and its momentum is rounding noise of the well-balanced eta - B (deep water)."""
    import numpy as np
    q_ref = np.asarray(q_ref)
    own = np.abs(q_ref).max(axis=tuple(range(1, q_ref.ndim)))
    out = own.astype(float).copy()
    for m in range(M):
        hmax = own[3 * m]
        phys = hmax * np.sqrt(g * hmax)
        out[3 * m + 1] = max(own[3 * m + 1], phys)
        out[3 * m + 2] = max(own[3 * m + 2], phys)
    return np.maximum(out, 1e-300)


def state_err(a, b, M, g=G, scale=None):
    """Per-field max |a - b| over state_scale(b) (or the given scale)."""
    import numpy as np
    a = np.asarray(a); b = np.asarray(b)
    sc = state_scale(b, M, g) if scale is None else scale
    return np.abs(a - b).max(axis=tuple(range(1, a.ndim))) / sc


def report(name, err):
    """Prints the achieved per-field errors (shown with pytest -s)."""
    import numpy as np
    print(f"PARITY {name} " + " ".join(f"{float(e):.2e}" for e in np.atleast_1d(err)))
