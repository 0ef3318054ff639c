"""Courant control of the AMR driver on the GPU against the oracle's (Sec. 2: the time
refinement keeps every level's Courant number below one; an attempt above cfl_max is
rejected, every level restored, and the step retaken in the next round with the time step
the usual rule gives from the speeds the rejected attempt measured).

The oversized step is forced the same way on both sides: the wave speeds the next time step
comes from are scaled down to 40 % (the GPU through its clock record, the oracle directly),
so the next attempt runs at about 2.2 times the Courant number the rule aims at.
"""
import numpy as np
import pytest

import oracle as O
from oracle.amr import OracleAMR
from paper_1803_01450_gb300 import inputs as I
from conftest import rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-11


def _gpu(pkg, n_members=1, levels=2, ratios=(2,), regrid=4):
    cfg = pkg.Config(M=2, dry_tol=1e-6, max_levels=levels, ratio=list(ratios) + [2] * 3, flag_tol=1e-3,
                     regrid_interval=regrid, n_buf=2, cluster_eff=0.7, min_side=16, max_side=64)
    H = pkg.Hierarchy(cfg, [(0.0, 0.0, 1.0, 1.0, 50, 50)] * n_members)
    nf = 50 * int(np.prod(ratios)) if levels > 1 else 50
    for m in range(n_members):
        H.set_bathymetry(m, -np.ones((nf, nf)))
    return H


def _oracle(levels=2, ratios=(2,)):
    P = O.params(M=2, dry_tol=1e-6)
    nf = 50 * int(np.prod(ratios)) if levels > 1 else 50
    return OracleAMR(P, (0, 0, 1, 1), 50, 50, levels, list(ratios) if levels > 1 else [], -np.ones((nf, nf)),
                     min_side=16, max_side=64)


def _scale_gpu_speeds(H, members, scale):
    c = H.get_clock()
    n, L = H.n_members, H.cfg.max_levels
    for m in members:
        for l in range(L):
            d = m * L + l
            c[n + 2 * d] *= scale
            c[n + 2 * d + 1] *= scale
    H.set_clock(c)


def _compare(H, A, member=0):
    assert abs(H.get_time()[0][member] - A.t) <= 1e-12 * A.t
    assert rel_err(H.get_state(member, 0), A.lev[0].q).max() < TOL
    for l in range(1, A.L):
        gp = [tuple(b) for b in H.get_patches(member, l).tolist()]
        assert gp == [tuple(b) for b in A.lev[l].patches]
        if gp:
            m = A.lev[l].in_patch_mask()
            assert rel_err(H.get_state(member, l)[:, m], A.lev[l].q[:, m]).max() < TOL


@pytest.mark.parametrize("levels,ratios", [(1, ()), (2, (2,)), (3, (2, 2))])
def test_forced_step_is_retaken_like_the_oracle(mlswe_lib, levels, ratios):
    w = I.small(50)
    H = _gpu(mlswe_lib, levels=levels, ratios=ratios)
    A = _oracle(levels, ratios)
    H.set_state(0, 0, w["q"])
    A.set_state(0, w["q"])
    H.advance(4)
    A.advance(4, regrid_interval=4)
    _scale_gpu_speeds(H, [0], 0.4)
    for l in range(A.L):
        A.smax[l] = A.smax[l] * 0.4
    H.advance(4)
    A.advance(4, regrid_interval=4)
    assert A.rejected == 1
    st = H.get_stats()
    assert st["cfl_exceeded"] == 1 and st["last_cfl"] <= 1.0
    _compare(H, A)
    # and the runs go on together
    H.advance(4)
    A.advance(4, regrid_interval=4)
    assert H.get_stats()["cfl_exceeded"] == 1 and A.rejected == 1
    _compare(H, A)
    H.close()


def test_only_the_forced_member_retakes(mlswe_lib):
    """Two members in one launch: member 1's oversized step is rejected and retaken in a
    round member 0 sits out; each member equals its own oracle run."""
    w = I.small(50)
    H = _gpu(mlswe_lib, n_members=2)
    A = [_oracle(), _oracle()]
    for m in range(2):
        H.set_state(m, 0, w["q"])
        A[m].set_state(0, w["q"])
    H.advance(4)
    for a in A:
        a.advance(4, regrid_interval=4)
    _scale_gpu_speeds(H, [1], 0.4)
    for l in range(2):
        A[1].smax[l] = A[1].smax[l] * 0.4
    H.advance(3)
    for a in A:
        a.advance(3, regrid_interval=4)
    assert A[0].rejected == 0 and A[1].rejected == 1
    assert H.get_stats()["cfl_exceeded"] == 1
    for m in range(2):
        _compare(H, A[m], m)
    H.close()


def test_graph_and_direct_launches_retake_alike(mlswe_lib):
    """The retake rounds replay the captured coarse-step graphs; direct launches give the same
    states bit for bit."""
    w = I.small(50)
    out = []
    for graphs in (True, False):
        H = _gpu(mlswe_lib)
        H.set_execution(use_graphs=graphs)
        H.set_state(0, 0, w["q"])
        H.advance(4)
        _scale_gpu_speeds(H, [0], 0.4)
        H.advance(4)
        out.append((H.get_state(0, 0), H.get_state(0, 1), H.get_time()[0], H.get_stats()["cfl_exceeded"]))
        H.close()
    (a0, a1, ta, ca), (b0, b1, tb, cb) = out
    assert ca == cb == 1 and np.array_equal(ta, tb)
    assert np.array_equal(a0, b0) and np.array_equal(a1, b1)
