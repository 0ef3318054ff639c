"""Subcycled AMR runs on the GPU against the oracle's, in configurations the other AMR tests do
not reach: one layer with ratios 2 then 4 on a non-square domain, three layers with ratio 4,
two layers with ratios 4 then 2 at first order over a shore whose lower layer ends inside the
refined region. Regrids every 3 coarse steps and automatic time steps. Patch layouts after
every regrid and the member time must be equal (integer and time-step decisions), every
level's patch cells within 1e-11 of the field scale (state_scale), and the composite layer
masses equal to 1e-12 (the reflux keeps them constant on both sides)."""
import numpy as np
import pytest

import oracle as O
from oracle.amr import OracleAMR
from conftest import report, state_err

pytestmark = pytest.mark.gpu
TOL = 1e-11
G = 9.81


def _hump(X, Y, x0=0.45, y0=0.5, a=0.02, w=0.006):
    return a * np.exp(-((X - x0) ** 2 + (Y - y0) ** 2) / w)


def _case(kind):
    """(M, rho, ratios, order, limiter, nx0, ny0, domain, B_finest, q0): states at rest except
    for a hump on the top surface; layers stacked under the surfaces eta_m (Eq. (4))."""
    if kind == "one_layer_2_4":
        M, rho, ratios, order, lim, nx0, ny0, dom = 1, (1000.0,), [2, 4], 2, 2, 24, 20, (0.0, 0.0, 1.2, 1.0)
        surfaces = [0.0]
        def bath(x, y): return -1.0 + 0.0 * x
    elif kind == "three_layers_4":
        M, rho, ratios, order, lim, nx0, ny0, dom = 3, (1000.0, 1020.0, 1030.0), [4], 2, 2, 24, 24, (0.0, 0.0, 1.0, 1.0)
        surfaces = [0.0, -0.3, -0.6]
        def bath(x, y): return -1.0 + 0.0 * x
    else:  # "two_layers_4_2_shore"
        M, rho, ratios, order, lim, nx0, ny0, dom = 2, (1000.0, 1025.0), [4, 2], 1, 0, 24, 24, (0.0, 0.0, 1.0, 1.0)
        surfaces = [0.0, -0.4]
        def bath(x, y): return np.where(x < 0.55, -1.0, -1.0 + 2.0 * (x - 0.55))  # reaches -0.4 at x = 0.85
    r = int(np.prod(ratios))
    nxf, nyf = nx0 * r, ny0 * r
    xf = dom[0] + (np.arange(nxf) + 0.5) * (dom[2] - dom[0]) / nxf
    yf = dom[1] + (np.arange(nyf) + 0.5) * (dom[3] - dom[1]) / nyf
    Xf, Yf = np.meshgrid(xf, yf)
    Bf = np.ascontiguousarray(bath(Xf, Yf))
    B0 = O.bathy_average(Bf, r)
    x = dom[0] + (np.arange(nx0) + 0.5) * (dom[2] - dom[0]) / nx0
    y = dom[1] + (np.arange(ny0) + 0.5) * (dom[3] - dom[1]) / ny0
    X, Y = np.meshgrid(x, y)
    eta = [np.full_like(B0, s) for s in surfaces]
    eta[0] = eta[0] + _hump(X, Y)
    q = np.zeros((3 * M, ny0, nx0))
    below = B0.copy()
    for m in range(M - 1, -1, -1):  # bottom layer first: h_m = max(0, eta_m - max(B, eta_{m+1}))
        h = np.maximum(eta[m] - below, 0.0)
        q[3 * m] = h
        below = below + h
    return M, rho, ratios, order, lim, nx0, ny0, dom, Bf, q


@pytest.mark.parametrize("kind", ["one_layer_2_4", "three_layers_4", "two_layers_4_2_shore"])
def test_amr_configuration_matches_oracle(mlswe_lib, kind):
    pkg = mlswe_lib
    M, rho, ratios, order, lim, nx0, ny0, dom, Bf, q = _case(kind)
    L = len(ratios) + 1
    cfg = pkg.Config(M=M, rho=rho, dry_tol=1e-6, order=order, limiter=lim, max_levels=L, ratio=ratios,
                     flag_tol=1e-3, regrid_interval=3, n_buf=2, cluster_eff=0.7, min_side=8, max_side=32)
    H = pkg.Hierarchy(cfg, [(dom[0], dom[1], dom[2], dom[3], nx0, ny0)])
    H.set_bathymetry(0, Bf)
    H.set_state(0, 0, q)
    P = O.params(M=M, rho=rho, dry_tol=1e-6, order=order, limiter=lim)
    A = OracleAMR(P, dom, nx0, ny0, L, ratios, Bf, flag_tol=1e-3, min_side=8, max_side=32)
    A.set_state(0, q)
    for _ in range(3):
        H.advance(3)
        A.advance(3, regrid_interval=3)
        for l in range(1, L):
            assert [tuple(b) for b in H.get_patches(0, l).tolist()] == [tuple(b) for b in A.lev[l].patches]
    assert len(A.lev[1].patches) > 0
    t, _ = H.get_time()
    assert abs(t[0] - A.t) <= 1e-12 * A.t
    err = state_err(H.get_state(0, 0), A.lev[0].q, M)
    for l in range(1, L):
        m = A.lev[l].in_patch_mask()
        if m.any():
            err = np.maximum(err, state_err(H.get_state(0, l)[:, m], A.lev[l].q[:, m], M))
    report(f"amr_config_{kind}", err)
    assert err.max() < TOL, err

    # composite masses (uncovered cells of every level), GPU against the oracle's
    gm = np.zeros(M)
    for l in range(L):
        V = A.lev[l]
        qg = H.get_state(0, l)
        m = V.in_patch_mask() if l > 0 else np.ones((V.ny, V.nx), bool)
        m = m & ~A.covered_mask(l)
        for k in range(M):
            gm[k] += qg[3 * k][m].sum() * V.dx * V.dy
    assert np.all(np.abs(gm - A.mass()) <= 1e-12 * A.mass())
    H.close()
