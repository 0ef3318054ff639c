"""Asynchronous input and gauge output (mlswe_set_state_async, mlswe_read_gauges_async,
mlswe_synchronize): the same values as the synchronous calls, in stream order with the
steps around them, through a pipelined loop whose next input is enqueued before the step
in flight finishes, and across staging buffers of growing size."""
import numpy as np
import pytest
import torch

from paper_1803_01450_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _pinned(a):
    t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True).numpy()
    t[...] = a
    return t


def _hier(pkg, n=64, levels=1):
    cfg = pkg.Config(M=2, dry_tol=1e-6, max_levels=levels, ratio=[2, 2, 2], min_side=8, max_side=32)
    H = pkg.Hierarchy(cfg, [(0.0, 0.0, 1.0, 1.0, n, n)])
    nf = n * 2 ** (levels - 1)
    H.set_bathymetry(0, -np.ones((nf, nf)))
    return H


def test_async_state_equals_sync_state(mlswe_lib):
    q, _ = I.gaussian_random_state(1, 2, 64, 64)
    H = _hier(mlswe_lib)
    H.set_state_async(0, 0, _pinned(q))
    H.synchronize()
    assert np.array_equal(H.get_state(0, 0), q)
    H.close()


def test_stream_order_with_steps(mlswe_lib):
    """A step enqueued before the asynchronous input reads the old state (its gauges say
    so); the state after it is the new input, bit for bit."""
    qa, B = I.gaussian_random_state(2, 2, 64, 64)
    qb, _ = I.gaussian_random_state(3, 2, 64, 64)
    xy = np.array([[0.3, 0.4], [0.7, 0.2]])
    ref = _hier(mlswe_lib)
    ref.set_bathymetry(0, -np.ones((64, 64)))
    ref.set_state(0, 0, qa)
    ref.step_level(0, dt=1e-4)
    g_ref = ref.read_gauges(0, xy)
    ref.close()
    H = _hier(mlswe_lib)
    H.set_state(0, 0, qa)
    H.set_dt(0, 1e-4)
    out = _pinned(np.zeros((2, 2)))
    H.step_level(0)
    H.read_gauges_async(0, xy, out)
    H.set_state_async(0, 0, _pinned(qb))
    H.synchronize()
    assert np.array_equal(out, g_ref)
    assert np.array_equal(H.get_state(0, 0), qb)
    H.close()


def test_pipelined_loop_matches_synchronous_loop(mlswe_lib):
    """Inputs cycling through three states, one step each, gauges after every step: the
    pipelined form (next input enqueued before waiting) gives the synchronous results."""
    states = [I.gaussian_random_state(s, 2, 80, 96)[0] for s in (4, 5, 6)]
    xy = np.stack([np.linspace(0.1, 0.9, 8), np.linspace(0.2, 0.8, 8)], axis=1)
    cfg = mlswe_lib.Config(M=2, dry_tol=1e-6, max_levels=1)

    def make():
        H = mlswe_lib.Hierarchy(cfg, [(0.0, 0.0, 1.0, 1.0, 80, 96)])
        H.set_bathymetry(0, -np.ones((96, 80)))
        H.set_dt(0, 1e-4)
        return H

    seq = [k % 3 for k in range(7)]
    H = make()
    sync_out = []
    for k in seq:
        H.set_state(0, 0, states[k])
        H.step_level(0)
        sync_out.append(H.read_gauges(0, xy))
    H.close()
    H = make()
    pinned = [_pinned(s) for s in states]
    outs = [_pinned(np.zeros((8, 2))) for _ in seq]
    H.set_state_async(0, 0, pinned[seq[0]])
    for k in range(len(seq)):
        H.step_level(0)
        H.read_gauges_async(0, xy, outs[k])
        if k + 1 < len(seq):
            H.set_state_async(0, 0, pinned[seq[k + 1]])
        H.synchronize()
    H.close()
    for a, b in zip(sync_out, outs):
        assert np.array_equal(a, b)


def test_staging_grows_with_the_level(mlswe_lib):
    """Level 0 then the (larger) level 1 of a two-level hierarchy through the same calls."""
    H = _hier(mlswe_lib, n=32, levels=2)
    q0, _ = I.gaussian_random_state(7, 2, 32, 32)
    q1, _ = I.gaussian_random_state(8, 2, 64, 64)
    H.set_state_async(0, 0, _pinned(q0))
    H.set_state_async(0, 1, _pinned(q1))
    H.set_state_async(0, 0, _pinned(q0 * 1.5))
    H.synchronize()
    assert np.array_equal(H.get_state(0, 0), q0 * 1.5)
    assert np.array_equal(H.get_state(0, 1), q1)
    H.close()


def test_bad_arguments(mlswe_lib):
    H = _hier(mlswe_lib)
    with pytest.raises(mlswe_lib.MLSWEError):
        H.set_state_async(0, 0, np.zeros((6, 10, 10)))
    with pytest.raises(mlswe_lib.MLSWEError):
        H.set_state_async(0, 3, np.zeros((6, 64, 64)))
    H.close()
