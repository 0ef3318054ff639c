"""Pins of the oracle's Courant-number control (Sec. 2: the time-refinement ratio exists to keep
every level's Courant number below one; an attempt above cfl_max is rejected and retaken).

* A step forced far above the limit (its time step taken from wave speeds scaled down to 40 %)
  is rejected, the retake is kept below cfl_max, and the time advances by the kept step only.
* The rejected attempt leaves nothing behind: the run equals, bit for bit, a run that never
  saw the oversized step and starts from the wave speeds the rejected attempt measured (so a
  level left unrestored, planted below, fails the pin).
* With the ordinary time-step rule nothing is rejected on the small workload, and every kept
  step of every run stays at or below cfl_max.
"""
import copy
import types

import numpy as np
import pytest

import oracle as O
from oracle.amr import OracleAMR
from paper_1803_01450_gb300 import inputs as I


def _small(levels=2, ratios=(2,)):
    w = I.small(50)
    P = O.params(M=2, dry_tol=1e-6)
    nf = 50 * int(np.prod(ratios))
    A = OracleAMR(P, (0, 0, 1, 1), 50, 50, levels, list(ratios), -np.ones((nf, nf)), min_side=16, max_side=64)
    A.set_state(0, w["q"])
    return A


def _forced(levels=2, ratios=(2,), scale=0.4):
    A = _small(levels, ratios)
    A.advance(2, regrid_interval=4)
    before = copy.deepcopy(A)
    for l in range(A.L):
        A.smax[l] = A.smax[l] * scale
    return A, before


def _same(A, B):
    for VA, VB in zip(A.lev, B.lev):
        if VA.patches != VB.patches or not np.array_equal(VA.q, VB.q):
            return False
    return A.t == B.t


@pytest.mark.parametrize("levels,ratios", [(2, (2,)), (3, (2, 2))])
def test_forced_step_rejected_and_retaken(levels, ratios):
    A, before = _forced(levels, ratios)
    t0, n_hist = A.t, len(A.history)
    A.advance(3)
    hist = A.history[n_hist:]
    assert A.rejected == 1 and not A.cfl_failed
    assert hist[0][1] is False and hist[0][0] > A.cfl_max
    assert all(c <= A.cfl_max for c, kept in hist if kept) and sum(k for _, k in hist) == 3
    assert A.t > t0


@pytest.mark.parametrize("levels,ratios", [(2, (2,)), (3, (2, 2))])
def test_rejected_attempt_leaves_nothing_behind(levels, ratios):
    A, before = _forced(levels, ratios)
    A.advance(3)
    B = before
    B.smax = [s.copy() for s in A.rejected_smax]
    B.advance(3)
    assert B.rejected == 0
    assert _same(A, B)


def test_planted_partial_restore_fails_the_pin():
    """A rejection that restores level 0 only (the refined level keeps what the rejected
    attempt wrote) no longer equals the run that never saw the oversized step."""
    A, before = _forced()

    def advance_keep_fine(self, n, regrid_interval=0, dt=None):
        done = 0
        while done < n:
            step_dt = self.next_dt()
            self.smax = [np.zeros(2) for _ in range(self.L)]
            self.level_dt = [0.0] * self.L
            saved0 = self.lev[0].q.copy()
            self.advance_level(0, step_dt, 0.0)
            self.dt = step_dt
            if self.courant() > self.cfl_max:
                self.lev[0].q = saved0  # planted: level 1 is not restored
                self.rejected += 1
                self.rejected_smax = [s.copy() for s in self.smax]
                continue
            self.t += step_dt
            done += 1

    A.advance = types.MethodType(advance_keep_fine, A)
    A.advance(1)
    assert A.rejected == 1
    before.smax = [s.copy() for s in A.rejected_smax]
    before.advance(1)
    assert not _same(A, before)


def test_no_rejection_with_the_usual_rule():
    A = _small()
    A.advance(40, regrid_interval=4)
    assert A.rejected == 0 and len(A.history) == 40
    assert max(c for c, _ in A.history) <= A.cfl_max


def test_retry_budget_gives_up_when_the_target_is_above_the_limit():
    """cfl_desired above cfl_max: every attempt is rejected; the run gives up after its
    budget of retake rounds with the state of its last kept step."""
    A = _small()
    A.advance(2, regrid_interval=4)
    q0 = A.lev[0].q.copy()
    t0 = A.t
    A.cfl = 1.5
    A.advance(2)
    assert A.cfl_failed and A.t == t0 and np.array_equal(A.lev[0].q, q0)
