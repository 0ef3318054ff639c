"""Pins of the oracle's unsplit step (wave propagation with transverse Riemann solves, the
corner-transport form): the transverse split against the transverse Jacobian and its
positive part built here with numpy; the step against facts that hold for any correct
corner-transport scheme: exact reduction to the split step on data that vary in x only,
exact symmetry under exchanging x and y (which dimensional splitting breaks), the exact
diagonal shift of the advective limit at unit Courant numbers in all four directions, lake
at rest, mass per layer, and a long run at Courant number 0.9 that stays bounded."""
import numpy as np
import pytest

import oracle as O

RHO3 = (1000.0, 1020.0, 1030.0)


def _roe(qL, qR, M):
    """Per layer: mean depth, Roe normal and transverse velocities (the edge state)."""
    hb, un, ut = np.zeros(M), np.zeros(M), np.zeros(M)
    for m in range(M):
        hL, hR = qL[3 * m], qR[3 * m]
        sl, sr = np.sqrt(hL), np.sqrt(hR)
        hb[m] = 0.5 * (hL + hR)
        un[m] = (sl * qL[3 * m + 1] / hL + sr * qR[3 * m + 1] / hR) / (sl + sr)
        ut[m] = (sl * qL[3 * m + 2] / hL + sr * qR[3 * m + 2] / hR) / (sl + sr)
    return hb, un, ut


def _transverse_jacobian(M, rho, g, hb, un, ut, coupled=True):
    """Jacobian of the transverse flux (ht, hn ht / h, ht^2 / h + g h^2 / 2 + coupling) per
    layer in the (h, hn, ht) order, at the edge state; the coupling adds g hbar_m C_mn to the
    h_n columns of the ht_m row (C_mn = 1 for n >= m, rho_n / rho_m for n < m)."""
    J = np.zeros((3 * M, 3 * M))
    for m in range(M):
        a = 3 * m
        J[a, a + 2] = 1.0
        J[a + 1, a] = -un[m] * ut[m]
        J[a + 1, a + 1] = ut[m]
        J[a + 1, a + 2] = un[m]
        J[a + 2, a] = -ut[m] ** 2
        J[a + 2, a + 2] = 2.0 * ut[m]
        for n in range(M):
            if n == m or coupled:
                J[a + 2, 3 * n] += g * hb[m] * (1.0 if n >= m else rho[n] / rho[m])
    return J


def _positive_part(J):
    lam, R = np.linalg.eig(J)
    lam, R = lam.real, R.real
    return R @ np.diag(np.maximum(lam, 0.0)) @ np.linalg.inv(R)


def _edge(rng, M, depths, ut_common=None, shear=0.0):
    q = []
    for _ in range(2):
        qs = np.zeros(3 * M)
        for m in range(M):
            h = depths[m] * (1.0 + 0.1 * rng.standard_normal())
            qs[3 * m] = h
            qs[3 * m + 1] = h * 0.1 * rng.standard_normal()
            v = ut_common if ut_common is not None else 0.1 * rng.standard_normal()
            qs[3 * m + 2] = h * (v + shear * rng.standard_normal())
        q.append(qs)
    return q[0], q[1]


@pytest.mark.parametrize("M, depths, rho", [(1, (1.3,), None), (2, (0.6, 0.4), (1000.0, 1025.0)),
                                            (3, (0.5, 0.3, 0.7), RHO3)])
def test_transverse_split_is_the_jacobian_split(M, depths, rho):
    """bp + bm = J_t dq, and bp = R max(Lambda, 0) R^-1 dq with the eigen-decomposition of the
    transverse Jacobian by numpy. With one transverse velocity in all layers (or one layer)
    the eigenvalue guesses are the roots, so both hold to rounding."""
    rng = np.random.default_rng(10 + M)
    P = O.params(M=M, rho=rho, dry_tol=1e-6)
    rr = rho if rho is not None else (1000.0,)
    for _ in range(40):
        v = 0.07 * rng.standard_normal()
        qL, qR = _edge(rng, M, depths, ut_common=v if M > 1 else None)
        if M > 1:  # equal transverse Roe velocities need equal transverse velocities per side
            for q in (qL, qR):
                q[2::3] = v * q[0::3]
        dq = rng.standard_normal(3 * M)
        bp, bm = O.transverse(P, qL, qR, -2.0, -2.0, dq)
        hb, un, ut = _roe(qL, qR, M)
        J = _transverse_jacobian(M, rr, 9.81, hb, un, ut)
        sc = np.abs(J).max() * np.abs(dq).max()
        assert np.abs(bp + bm - J @ dq).max() <= 1e-12 * sc
        assert np.abs(bp - _positive_part(J) @ dq).max() <= 1e-11 * sc


def test_transverse_split_with_shear_between_layers():
    """Different transverse velocities per layer: the two Newton steps leave an eigenvalue
    error of order du^4 relative to the internal speeds (below 1e-9 here)."""
    rng = np.random.default_rng(21)
    P = O.params(M=2, dry_tol=1e-6)
    for _ in range(40):
        qL, qR = _edge(rng, 2, (0.6, 0.4), ut_common=0.02, shear=0.002)
        dq = rng.standard_normal(6)
        bp, bm = O.transverse(P, qL, qR, -2.0, -2.0, dq)
        hb, un, ut = _roe(qL, qR, 2)
        J = _transverse_jacobian(2, (1000.0, 1025.0), 9.81, hb, un, ut)
        sc = np.abs(J).max() * np.abs(dq).max()
        assert np.abs(bp + bm - J @ dq).max() <= 1e-9 * sc
        assert np.abs(bp - _positive_part(J) @ dq).max() <= 1e-8 * sc


def test_transverse_split_of_a_decoupled_edge():
    """Lower layer dry on one side: each layer is split alone (no coupling), the layer that
    is wet on one side only with its Roe state, the both-dry layer sends nothing."""
    rng = np.random.default_rng(22)
    P = O.params(M=2, dry_tol=1e-6)
    for _ in range(20):
        qL, qR = _edge(rng, 2, (0.6, 0.4))
        qR[3:6] = 0.0  # layer 2 dry on the right; its surface lies above the dry side's bed
        dq = rng.standard_normal(6)
        bp, bm = O.transverse(P, qL, qR, -1.0, -0.7, dq)
        hb, un, ut = _roe(qL, qR, 1)
        J1 = _transverse_jacobian(1, (1000.0,), 9.81, hb, un, ut)
        sc = np.abs(dq).max() * 10
        assert np.abs((bp + bm)[:3] - J1 @ dq[:3]).max() <= 1e-12 * sc
        assert np.abs(bp[:3] - _positive_part(J1) @ dq[:3]).max() <= 1e-11 * sc
        # layer 2 (wet on the left only) flows onto the dry cell: Roe state with sqrt(0) = 0
        h2 = qL[3]
        hb2, un2, ut2 = 0.5 * h2, qL[4] / h2, qL[5] / h2
        J2 = _transverse_jacobian(1, (1000.0,), 9.81, [hb2], [un2], [ut2])
        assert np.abs((bp + bm)[3:] - J2 @ dq[3:]).max() <= 1e-12 * sc
        assert np.abs(bp[3:] - _positive_part(J2) @ dq[3:]).max() <= 1e-11 * sc
        qL[3:6] = 0.0  # both dry: nothing
        bp, bm = O.transverse(P, qL, qR, -1.0, -0.7, dq)
        assert not bp[3:].any() and not bm[3:].any()


def _grid(n):
    x = (np.arange(n) + 0.5) / n
    return np.meshgrid(x, x)


def _layered(M, X, Y, B, hump=0.03, vel=0.05):
    surf = {1: [0.0], 2: [0.0, -0.4], 3: [0.0, -0.3, -0.6]}[M]
    q = np.zeros((3 * M,) + X.shape)
    lower = B.copy()
    for m in range(M - 1, -1, -1):
        s = surf[m] + (hump * np.exp(-((X - 0.4) ** 2 + (Y - 0.6) ** 2) / 0.01) if m == 0 else 0.0)
        top = np.maximum(s, lower)
        q[3 * m] = top - lower
        lower = top
        q[3 * m + 1] = q[3 * m] * vel * np.sin(2 * X + Y + m)
        q[3 * m + 2] = q[3 * m] * vel * np.cos(X - 2 * Y + m)
    return q


@pytest.mark.parametrize("M", [1, 2])
@pytest.mark.parametrize("order", [1, 2])
def test_unsplit_equals_split_on_data_varying_in_x_only(M, order):
    """With no y variation the y edges carry no waves and the transverse corrections of the
    edges above and below a cell are equal: the step is the x sweep alone."""
    n = 24
    X, Y = _grid(n)
    B = -1.0 + 0.3 * np.exp(-(X - 0.5) ** 2 / 0.02) + 0.0 * Y
    q = np.zeros((3 * M, n, n))
    if M == 1:
        q[0] = 0.02 * np.exp(-(X - 0.3) ** 2 / 0.01) - B
        q[1] = 0.05 * q[0] * np.sin(3 * X)
    else:
        q[3] = np.maximum(-0.4 - B, 0.0)
        q[0] = 0.02 * np.exp(-(X - 0.3) ** 2 / 0.01) + 0.4
        q[1] = 0.02 * q[0] * np.sin(3 * X)
        q[4] = -0.01 * q[3] * np.cos(2 * X)
    dt = 0.4 / n / 3.2
    a, _, _ = O.step_walled(O.params(M=M, dry_tol=1e-6, order=order), q, B, 1 / n, 1 / n, dt)
    b, _, _ = O.step_walled(O.params(M=M, dry_tol=1e-6, order=order, unsplit=1), q, B, 1 / n, 1 / n, dt)
    assert np.abs(a - b).max() <= 1e-15 * np.abs(a).max()
    assert not b[2::3].any()  # no y momentum appears


@pytest.mark.parametrize("M, rho", [(1, None), (2, None), (3, RHO3)])
def test_unsplit_is_symmetric_under_exchanging_x_and_y(M, rho):
    """Transposing the state (and exchanging hu, hv) and the bathymetry commutes with the
    unsplit step up to rounding; dimensional splitting (x first) breaks it at O(dt^2)."""
    n = 24
    X, Y = _grid(n)
    B = -1.0 + 0.2 * np.sin(2 * np.pi * X) * np.cos(3 * np.pi * Y) + 0.1 * X * Y
    q = _layered(M, X, Y, B)
    dt = 0.5 / n / 3.2

    def swap(a):
        b = np.transpose(a, (0, 2, 1)).copy()
        for m in range(M):
            b[[3 * m + 1, 3 * m + 2]] = b[[3 * m + 2, 3 * m + 1]]
        return b

    for unsplit in (0, 1):
        P = O.params(M=M, rho=rho, dry_tol=1e-6, unsplit=unsplit)
        a, _, _ = O.step_walled(P, q, B, 1 / n, 1 / n, dt)
        b, _, _ = O.step_walled(P, swap(q), B.T.copy(), 1 / n, 1 / n, dt)
        d = np.abs(a - swap(b)).max() / np.abs(a).max()
        if unsplit:
            assert d <= 1e-14
        else:
            assert d > 1e-6


@pytest.mark.parametrize("M", [1, 2])
@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("U, V", [(1.0, 1.0), (-1.0, 1.0), (1.0, -1.0), (-1.0, -1.0)])
def test_advective_limit_at_unit_courant_numbers_shifts_exactly(M, order, U, V):
    """As g -> 0 every layer is carried by the uniform velocity (U, V); with dt = dx / |U| =
    dy / |V| the corner-transport step moves every cell one cell diagonally, exactly (the
    property that needs the transverse corrections: without them, or with a wrong sign,
    factor or receiving cell, the result is off by O(1) of the bump). Remaining error: of
    the order of the gravity speed sqrt(g h) = 1e-8 relative to |U|, amplified by the
    near-coincident wave speeds."""
    n = 32
    X, Y = _grid(n)
    B = -np.ones((n, n)) * (2.0 if M == 2 else 1.0)
    bump = 0.3 * np.exp(-((X - 0.45) ** 2 + (Y - 0.5) ** 2) / 0.01)
    q = np.zeros((3 * M, n, n))
    q[0] = 1.0 + bump
    if M == 2:
        q[3] = 1.0
    for m in range(M):
        q[3 * m + 1] = U * q[3 * m]
        q[3 * m + 2] = V * q[3 * m]
    P = O.params(M=M, g=1e-16, dry_tol=1e-6, order=order, unsplit=1)
    a, _, _ = O.step_walled(P, q, B, 1 / n, 1 / n, 1 / n)
    ref = np.roll(np.roll(q, int(np.sign(V)), axis=1), int(np.sign(U)), axis=2)
    s = slice(4, n - 4)  # away from the walls
    assert np.abs(a[:, s, s] - ref[:, s, s]).max() <= 1e-8 * 0.3


@pytest.mark.parametrize("M, rho", [(1, None), (2, None), (3, RHO3)])
def test_unsplit_lake_at_rest_and_mass(M, rho):
    n = 24
    X, Y = _grid(n)
    B = -1.5 + 0.4 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)
    rest = _layered(M, X, Y, B, hump=0.0, vel=0.0)
    for order in (1, 2):
        P = O.params(M=M, rho=rho, dry_tol=1e-6, order=order, unsplit=1)
        qn = rest.copy()
        for _ in range(5):
            qn, _, _ = O.step_walled(P, qn, B, 1 / n, 1 / n, 0.3 / n / 4.0)
        assert np.abs(qn - rest).max() <= 1e-13
    q = _layered(M, X, Y, B)
    P = O.params(M=M, rho=rho, dry_tol=1e-6, unsplit=1)
    qn = q.copy()
    for _ in range(10):
        qn, _, lost = O.step_walled(P, qn, B, 1 / n, 1 / n, 0.3 / n / 4.0)
    for m in range(M):
        assert abs(qn[3 * m].sum() - q[3 * m].sum()) <= 1e-13 * q[3 * m].sum()


def test_unsplit_long_run_at_courant_number_09_stays_bounded():
    """Two layers, a hump on a sloping bed, 300 steps at Courant number 0.9 (time step from
    the previous step's speeds): the surface stays within the initial range plus a margin
    and every depth stays finite and non-negative."""
    n = 40
    X, Y = _grid(n)
    B = -1.0 + 0.2 * X
    q = _layered(2, X, Y, B, hump=0.05, vel=0.0)
    P = O.params(M=2, dry_tol=1e-6, unsplit=1)
    dt = 0.9 / n / np.sqrt(9.81 * 1.05)
    qn = q.copy()
    for _ in range(300):
        qn, smax, _ = O.step_walled(P, qn, B, 1 / n, 1 / n, dt)
        dt = 0.9 / n / max(smax)
    eta = B + qn[3] + qn[0]
    assert np.isfinite(qn).all() and qn[0].min() >= 0 and qn[3].min() >= 0
    assert np.abs(eta).max() <= 0.05
