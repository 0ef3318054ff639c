"""Failure detection, injected on the host (no GPU fault, trap or hang): every C-ABI call
reports what went wrong through its status code and leaves the hierarchy usable or cleanly
released. Cases: a non-finite state, a time step above the Courant limit, patch tables that
break nesting, allocation failures in the allocator callback, and a state with negative
depths (repaired by the positivity rule, not an error). Also: checkpoint and resume of a
subcycled AMR run through the public calls, bit for bit, and the run counters."""
import numpy as np
import pytest

from paper_1803_01450_gb300 import inputs as I

pytestmark = pytest.mark.gpu

OK, EINVAL, ENOMEM, ECUDA, ECFL, ENEGDEPTH, ENESTING = 0, 1, 2, 3, 4, 5, 6


def _small(pkg, levels=1, regrid=0, **kw):
    opts = dict(M=2, dry_tol=1e-6, max_levels=levels, ratio=[2, 2, 2], flag_tol=1e-3, regrid_interval=regrid,
                n_buf=2, cluster_eff=0.7, min_side=8, max_side=64)
    opts.update(kw)
    cfg = pkg.Config(**opts)
    H = pkg.Hierarchy(cfg, [(0.0, 0.0, 1.0, 1.0, 50, 50)])
    nf = 50 * 2 ** (levels - 1)
    H.set_bathymetry(0, -np.ones((nf, nf)))
    return H


def _raises(pkg, status, fn, *a, **k):
    with pytest.raises(pkg.MLSWEError) as e:
        fn(*a, **k)
    assert e.value.status == status, (e.value.status, str(e.value))


def test_non_finite_state_is_reported(mlswe_lib):
    w = I.small(50)
    q = w["q"].copy()
    q[0, 20, 20] = np.nan
    H = _small(mlswe_lib)
    H.set_state(0, 0, q)
    _raises(mlswe_lib, ENEGDEPTH, H.step_level, 0, dt=1e-3, want_cfl=True)
    H.set_state(0, 0, q)
    _raises(mlswe_lib, ENEGDEPTH, H.advance, 1)
    # the hierarchy stays usable with a finite state
    H.set_state(0, 0, w["q"])
    H.advance(2)
    assert np.isfinite(H.get_state(0, 0)).all()
    H.close()


def test_courant_number_above_limit_is_reported(mlswe_lib):
    """A level step above cfl_max (with a Courant report) is undone and reported; automatic
    steps aimed above cfl_max are rejected in every retake and the call gives up with the
    state of the last kept step."""
    w = I.small(50)
    H = _small(mlswe_lib)
    H.set_state(0, 0, w["q"])
    dt_ok = 0.9 * w["dx"] / 3.2
    cfl = H.step_level(0, dt=dt_ok, want_cfl=True)
    assert 0 < cfl[0] < 1.0
    q1 = H.get_state(0, 0)
    _raises(mlswe_lib, ECFL, H.step_level, 0, dt=10 * dt_ok, want_cfl=True)
    assert np.array_equal(H.get_state(0, 0), q1)  # undone
    H.close()
    # automatic time steps aimed above cfl_max: 2 rounds + 2 + 8 retake rounds, all rejected
    H = _small(mlswe_lib, cfl_desired=1.5, cfl_max=1.0)
    H.set_state(0, 0, w["q"])
    _raises(mlswe_lib, ECFL, H.advance, 2)
    st = H.get_stats()
    assert st["cfl_exceeded"] == 12 and st["last_cfl"] > 1.0
    assert np.array_equal(H.get_state(0, 0), w["q"]) and H.get_time()[0][0] == 0.0
    H.close()


def test_patch_tables_that_break_nesting_are_rejected(mlswe_lib):
    w = I.small(50)
    H = _small(mlswe_lib, levels=3)
    H.set_state(0, 0, w["q"])
    # level 1 (100 x 100): overlapping boxes, a box leaving the domain
    _raises(mlswe_lib, ENESTING, H.set_patches, 0, 1, np.array([[8, 8, 40, 40], [32, 32, 60, 60]]))
    _raises(mlswe_lib, ENESTING, H.set_patches, 0, 1, np.array([[80, 80, 120, 120]]))
    good = np.array([[8, 8, 40, 40], [48, 8, 80, 40]])
    H.set_patches(0, 1, good)
    # level 2 (200 x 200): a box outside every level-1 patch, one inside without the margin
    _raises(mlswe_lib, ENESTING, H.set_patches, 0, 2, np.array([[120, 120, 160, 160]]))
    _raises(mlswe_lib, ENESTING, H.set_patches, 0, 2, np.array([[16, 16, 48, 48]]))
    H.set_patches(0, 2, np.array([[24, 24, 56, 56]]))
    assert np.array_equal(H.get_patches(0, 1), good)
    H.interp_fine(0, 0)
    H.interp_fine(1, 0)
    H.advance(2)  # still usable
    assert np.isfinite(H.get_state(0, 0)).all()
    H.close()


class _FailingAllocator:
    """torch's caching allocator behind a switch: allocations fail once `budget` is spent."""

    def __init__(self, budget):
        import torch
        self.torch = torch
        self.dev = torch.cuda.current_device()
        self.budget = budget
        self.live = {}

    def alloc(self, nbytes):
        if self.budget <= 0:
            return 0
        self.budget -= 1
        p = self.torch.cuda.caching_allocator_alloc(nbytes, self.dev, 0)
        self.live[p] = nbytes
        return p

    def free(self, p):
        self.torch.cuda.caching_allocator_delete(p)
        del self.live[p]


def test_allocation_failures_are_reported_and_released(mlswe_lib):
    cfg = mlswe_lib.Config(M=2, dry_tol=1e-6, max_levels=2, ratio=[2], order=1)
    dom = [(0.0, 0.0, 1.0, 1.0, 40, 40)]
    for budget in (0, 3, 9):  # failing at the first, fourth and tenth allocation of creation
        a = _FailingAllocator(budget)
        with pytest.raises(mlswe_lib.MLSWEError) as e:
            mlswe_lib.Hierarchy(cfg, dom, allocator=(a.alloc, a.free))
        assert e.value.status == ENOMEM
        assert not a.live  # everything obtained before the failure was given back
    # creation succeeds, a later allocation (the adjoint's buffers) fails
    a = _FailingAllocator(10 ** 6)
    cfg1 = mlswe_lib.Config(M=2, dry_tol=1e-6, max_levels=1, order=1)
    H = mlswe_lib.Hierarchy(cfg1, dom, allocator=(a.alloc, a.free))
    q, B = I.gaussian_random_state(3, 2, 40, 40)
    H.set_bathymetry(0, B)
    H.set_state(0, 0, q)
    H.set_dt(0, 1e-4)
    a.budget = 2
    _raises(mlswe_lib, ENOMEM, H.adjoint_setup, 10, 5, np.array([[3, 4]]), np.zeros((10, 1)))
    a.budget = 10 ** 6
    H.step_level(0, dt=1e-4)  # still usable
    H.close()
    assert not a.live


def test_negative_depths_are_repaired_not_reported(mlswe_lib):
    q, B = I.gaussian_random_state(4, 2, 40, 40)
    q[0, 10:12, 10:12] = -0.05  # upper layer below zero in a few cells
    cfg = mlswe_lib.Config(M=2, dry_tol=1e-6, max_levels=1)
    H = mlswe_lib.Hierarchy(cfg, [(0.0, 0.0, 1.0, 1.0, 40, 40)])
    H.set_bathymetry(0, B)
    H.set_state(0, 0, q)
    H.step_level(0, dt=1e-4, want_cfl=True)
    out = H.get_state(0, 0)
    assert np.isfinite(out).all()
    assert out[0].min() >= 0.0 and out[3].min() >= 0.0
    H.close()


def test_checkpoint_and_resume_bit_for_bit(mlswe_lib):
    """Save the patch layout, the states of both levels and the clock after 6 coarse steps
    of a regridding two-level run; a new hierarchy restored from them continues exactly like
    the original (regrids included)."""
    w = I.small(50)
    A = _small(mlswe_lib, levels=2, regrid=4, min_side=16)
    A.set_state(0, 0, w["q"])
    A.advance(6)
    snap = (A.get_patches(0, 1), A.get_state(0, 0), A.get_state(0, 1), A.get_clock())
    A.advance(5)
    B = _small(mlswe_lib, levels=2, regrid=4, min_side=16)
    B.set_patches(0, 1, snap[0])
    B.set_state(0, 0, snap[1])
    B.set_state(0, 1, snap[2])
    B.set_clock(snap[3])
    B.advance(5)
    pa, pb = A.get_patches(0, 1), B.get_patches(0, 1)
    assert np.array_equal(pa, pb)
    assert np.array_equal(A.get_time()[0], B.get_time()[0])
    assert np.array_equal(A.get_state(0, 0), B.get_state(0, 0))
    m = np.zeros((100, 100), bool)
    for (i0, j0, i1, j1) in pa.tolist():
        m[j0:j1, i0:i1] = True
    assert np.array_equal(A.get_state(0, 1)[:, m], B.get_state(0, 1)[:, m])
    A.close()
    B.close()


def test_run_counters(mlswe_lib):
    w = I.small(50)
    H = _small(mlswe_lib, levels=2, regrid=4, min_side=16)
    H.set_state(0, 0, w["q"])
    H.advance(8)
    st = H.get_stats()
    assert st["coarse_steps"] == 8 and st["regrids"] == 2  # before coarse steps 0 and 4
    assert st["level_steps"] == [8, 16]  # ratio 2 subcycling
    assert st["cell_updates"][0] == 8 * 50 * 50
    assert st["cell_updates"][1] > 0 and st["cell_updates"][1] % 2 == 0
    assert st["patches"] == [1, H.get_patches(0, 1).shape[0]]
    assert st["cfl_exceeded"] == 0 and 0.5 < st["last_cfl"] < 1.0
    H.step_level(0, dt=1e-4)
    st2 = H.get_stats()
    assert st2["level_steps"] == [9, 16] and st2["cell_updates"][0] == 9 * 50 * 50
    H.close()
