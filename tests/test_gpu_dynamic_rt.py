"""Dynamic time-refinement ratio (Sec. 2: GeoClaw picks r_t per level and step, smaller where
the refined region is shallow) on the GPU against the oracle: patch layouts, time steps and
the number of steps per level (integer decisions: equal), states within 1e-11. An ensemble
whose members choose different ratios runs them in the same launches (members with fewer
substeps copy their state through the extra ones); each member matches its own oracle run."""
import numpy as np
import pytest

import oracle as O
from oracle.amr import OracleAMR
from conftest import rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-11


def _basin(n, r, shallow_east=True):
    """Basin on n x n coarse cells, bathymetry at n * r per side (r: the product of the ratios)."""
    nf = n * r
    xf = (np.arange(nf) + 0.5) / nf
    Xf, _ = np.meshgrid(xf, xf)
    if shallow_east:
        Bf = np.where(Xf < 0.5, -1.0, -0.05)
    else:
        Bf = -1.0 + 0.0 * Xf
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x)
    B0 = O.bathy_average(Bf, r)
    eta1 = 0.004 * np.exp(-((X - 0.75) ** 2 + (Y - 0.5) ** 2) / 0.004)
    q = np.zeros((6, n, n))
    q[3] = np.maximum(-0.02 - B0, 0.0)
    q[0] = eta1 - np.maximum(-0.02, B0)
    return Bf, q


def _gpu(pkg, members, n, r, dynamic):
    ratios = list(r) if isinstance(r, (list, tuple)) else [r]
    cfg = pkg.Config(M=2, rho=(1000.0, 1025.0), dry_tol=1e-6, max_levels=len(ratios) + 1, ratio=ratios, flag_tol=2e-3,
                     regrid_interval=4, n_buf=2, cluster_eff=0.7, min_side=8, max_side=32, dynamic_rt=dynamic)
    H = pkg.Hierarchy(cfg, [(0.0, 0.0, 1.0, 1.0, n, n)] * len(members))
    for k, (Bf, q) in enumerate(members):
        H.set_bathymetry(k, Bf)
        H.set_state(k, 0, q)
    return H


def _oracle(Bf, q, n, r, dynamic):
    ratios = list(r) if isinstance(r, (list, tuple)) else [r]
    A = OracleAMR(O.params(M=2, rho=(1000.0, 1025.0), dry_tol=1e-6), (0, 0, 1, 1), n, n, len(ratios) + 1, ratios, Bf,
                  flag_tol=2e-3, min_side=8, max_side=32, dynamic_rt=dynamic)
    A.set_state(0, q)
    return A


def _compare(H, k, A):
    assert rel_err(H.get_state(k, 0), A.lev[0].q).max() < TOL
    for l in range(1, A.L):
        assert [tuple(b) for b in H.get_patches(k, l).tolist()] == [tuple(b) for b in A.lev[l].patches]
        m = A.lev[l].in_patch_mask()
        if m.any():
            assert rel_err(H.get_state(k, l)[:, m], A.lev[l].q[:, m]).max() < TOL


def test_dynamic_time_ratio_matches_oracle(mlswe_lib):
    n, r, steps = 32, 4, 12
    Bf, q = _basin(n, r)
    H = _gpu(mlswe_lib, [(Bf, q)], n, r, 1)
    A = _oracle(Bf, q, n, r, True)
    for _ in range(steps // 4):
        H.advance(4)
        A.advance(4, regrid_interval=4)
        _compare(H, 0, A)
    t, dt = H.get_time()
    assert abs(t[0] - A.t) <= 1e-12 * A.t
    st = H.get_stats()
    assert st["level_steps"] == A.level_steps, (st["level_steps"], A.level_steps)
    assert st["level_steps"][1] < r * steps  # the shallow fine level took fewer steps
    H.close()


def test_three_levels_dynamic_time_ratio_matches_oracle(mlswe_lib):
    """Both refined levels choose their ratio (level 2 within each level-1 substep)."""
    n, r, steps = 24, (2, 2), 8
    Bf, q = _basin(n, 4)
    H = _gpu(mlswe_lib, [(Bf, q)], n, r, 1)
    A = _oracle(Bf, q, n, r, True)
    for _ in range(steps // 4):
        H.advance(4)
        A.advance(4, regrid_interval=4)
        _compare(H, 0, A)
    assert H.get_stats()["level_steps"] == A.level_steps, (H.get_stats()["level_steps"], A.level_steps)
    assert A.lev[2].patches and A.level_steps[2] < 4 * steps
    assert abs(H.get_time()[0][0] - A.t) <= 1e-12 * A.t
    H.close()


def test_members_with_different_time_ratios_share_launches(mlswe_lib):
    """Member 0 refines shallow water (small r_t), member 1 deep water (r_t = r): the launches
    run r substeps, member 0 copies its state through those beyond its r_t."""
    n, r, steps = 32, 4, 8
    members = [_basin(n, r, shallow_east=True), _basin(n, r, shallow_east=False)]
    H = _gpu(mlswe_lib, members, n, r, 1)
    As = [_oracle(Bf, q, n, r, True) for (Bf, q) in members]
    for _ in range(steps // 4):
        H.advance(4)
        for A in As:
            A.advance(4, regrid_interval=4)
        for k, A in enumerate(As):
            _compare(H, k, A)
    t, _ = H.get_time()
    for k, A in enumerate(As):
        assert abs(t[k] - A.t) <= 1e-12 * A.t
    assert As[0].level_steps[1] < As[1].level_steps[1]  # the members did choose differently
    st = H.get_stats()
    assert st["level_steps"][1] == max(A.level_steps[1] for A in As)
    H.close()


def test_fixed_ratio_unchanged_by_the_option(mlswe_lib):
    """dynamic_rt = 0 runs r substeps on every member, as before the option existed."""
    n, r, steps = 32, 4, 8
    Bf, q = _basin(n, r)
    H = _gpu(mlswe_lib, [(Bf, q)], n, r, 0)
    A = _oracle(Bf, q, n, r, False)
    H.advance(steps)
    A.advance(steps, regrid_interval=4)
    _compare(H, 0, A)
    assert H.get_stats()["level_steps"] == [steps, r * steps] == A.level_steps
    H.close()
