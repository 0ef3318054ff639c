"""Pins of the oracle's general M-layer coupled branch (M = 3 and 4, and M = 2 through the
same code): against the dedicated two-layer branch, the flux jumps written out from the PDE,
the eigenvectors of the Roe-state Jacobian built here with numpy, and the invariants of the
step (lake at rest, mass per layer, mirror symmetry)."""
import numpy as np
import pytest

import oracle as O

RHO3 = (1000.0, 1020.0, 1030.0)
RHO4 = (1000.0, 1020.0, 1030.0, 1040.0)
RHO = {3: RHO3, 4: RHO4}
# layer thicknesses (top first) at unit and ocean scales
DEPTHS = {3: [(0.5, 0.3, 0.7), (150.0, 600.0, 3200.0)], 4: [(0.4, 0.3, 0.35, 0.6), (100.0, 300.0, 800.0, 2800.0)]}


def _random_edge(rng, M, depths, vel=0.05, tr=0.05):
    q = []
    for side in range(2):
        qs = np.zeros(3 * M)
        for m in range(M):
            h = depths[m] * (1.0 + 0.1 * rng.standard_normal())
            qs[3 * m] = h
            qs[3 * m + 1] = h * vel * rng.standard_normal()
            qs[3 * m + 2] = h * tr * rng.standard_normal()
        q.append(qs)
    B = -sum(depths) + 0.05 * rng.standard_normal(2)
    return q[0], q[1], B[0], B[1]


def _flux_jumps(M, rho, g, qL, qR, BL, BR):
    """d0_m = D(hu), d1_m = D(hu u) + g hbar_m (D eta_m + sum_{n<m} rho_n/rho_m D h_n),
    d2_m = D(hu v): the PDE's normal flux jumps with the layer coupling folded in."""
    d = np.zeros((M, 3))
    hL, hR = qL[0::3], qR[0::3]
    etaL = BL + np.cumsum(hL[::-1])[::-1]
    etaR = BR + np.cumsum(hR[::-1])[::-1]
    for m in range(M):
        uL, uR = qL[3 * m + 1] / hL[m], qR[3 * m + 1] / hR[m]
        vL, vR = qL[3 * m + 2] / hL[m], qR[3 * m + 2] / hR[m]
        hb = 0.5 * (hL[m] + hR[m])
        coup = (etaR[m] - etaL[m]) + sum(rho[n] / rho[m] * (hR[n] - hL[n]) for n in range(m))
        d[m, 0] = qR[3 * m + 1] - qL[3 * m + 1]
        d[m, 1] = (qR[3 * m + 1] * uR - qL[3 * m + 1] * uL) + g * hb * coup
        d[m, 2] = qR[3 * m + 1] * vR - qL[3 * m + 1] * vL
    return d


def _roe_jacobian(M, rho, g, qL, qR):
    """Normal 2M x 2M Jacobian of ((h_m, hu_m))_m at the Roe state (Roe velocities, mean
    depths), with the coupling g h_m sum_n C_mn dh_n, C_mn = 1 (n >= m), rho_n/rho_m (n < m)."""
    J = np.zeros((2 * M, 2 * M))
    for m in range(M):
        hL, hR = qL[3 * m], qR[3 * m]
        u = (np.sqrt(hL) * qL[3 * m + 1] / hL + np.sqrt(hR) * qR[3 * m + 1] / hR) / (np.sqrt(hL) + np.sqrt(hR))
        hb = 0.5 * (hL + hR)
        J[2 * m, 2 * m + 1] = 1.0
        J[2 * m + 1, 2 * m] = -u * u
        J[2 * m + 1, 2 * m + 1] = 2.0 * u
        for n in range(M):
            J[2 * m + 1, 2 * n] += g * hb * (1.0 if n >= m else rho[n] / rho[m])
    return J


def test_general_branch_equals_two_layer_branch(orc):
    """At M = 2 the general coupled branch (Jacobi guesses, Newton on det, eigenvectors from
    the first rows, elimination) gives the waves of the dedicated two-layer branch."""
    rng = np.random.default_rng(1)
    P = orc.params(M=2, dry_tol=1e-6)
    for _ in range(200):
        qL, qR, BL, BR = _random_edge(rng, 2, (0.6, 0.4))
        Z, s, am, ap, info = orc.riemann(P, qL, qR, BL, BR)
        Zg, sg, amg, apg, infog = orc.riemann(P, qL, qR, BL, BR, general=True)
        assert np.array_equal(info, infog)
        sc = np.abs(s).max()
        assert np.abs(s - sg).max() <= 1e-13 * sc
        assert np.abs(am - amg).max() <= 1e-12 * max(np.abs(am).max(), 1e-300)
        assert np.abs(ap - apg).max() <= 1e-12 * max(np.abs(ap).max(), 1e-300)


@pytest.mark.parametrize("M,k", [(3, 0), (3, 1), (4, 0), (4, 1)])
def test_multilayer_waves_sum_to_flux_jumps(orc, M, k):
    depths = DEPTHS[M][k]
    rng = np.random.default_rng(2)
    P = orc.params(M=M, rho=RHO[M], dry_tol=1e-6)
    for _ in range(100):
        qL, qR, BL, BR = _random_edge(rng, M, depths)
        Z, s, am, ap, info = orc.riemann(P, qL, qR, BL, BR)
        assert info[-1] == 0
        d = _flux_jumps(M, RHO[M], 9.81, qL, qR, BL, BR)
        tot = Z.sum(axis=0).reshape(M, 3)
        sc = np.abs(d).max(axis=0)
        assert np.all(np.abs(tot - d) <= 1e-11 * sc), (tot, d)
        # fluctuations: A-dQ + A+dQ equals the jumps too
        assert np.all(np.abs((am + ap).reshape(M, 3) - d) <= 1e-11 * sc)


@pytest.mark.parametrize("M", [3, 4])
def test_multilayer_waves_are_jacobian_eigenvectors(orc, M):
    """Each acoustic wave (mass_m, lambda mass_m)_m is an eigenvector of the Roe-state
    Jacobian; its speed is an eigenvalue (numpy), exactly when the layers move together
    (the guesses are then the roots) and to the accuracy of two Newton steps otherwise (an
    error of order du^4 from guesses off by du: with shear speeds du ~ 0.002 against internal
    wave speeds ~ 0.1, below 1e-9 of the largest speed). Four layers put internal speeds
    0.004 apart, so their shear is halved to keep the guesses within Newton's reach."""
    rng = np.random.default_rng(3)
    P = orc.params(M=M, rho=RHO[M], dry_tol=1e-6)
    N = 2 * M
    du = {3: 0.002, 4: 0.001}[M]
    for equal in (True, False):
        for _ in range(50):
            qL, qR, BL, BR = _random_edge(rng, M, DEPTHS[M][0], vel=0.0 if equal else du)
            if equal:  # one common velocity in every layer and on both sides
                u = 0.03
                for q in (qL, qR):
                    q[1::3] = u * q[0::3]
            Z, s, am, ap, info = orc.riemann(P, qL, qR, BL, BR)
            J = _roe_jacobian(M, RHO[M], 9.81, qL, qR)
            ev = np.sort(np.linalg.eigvals(J).real)
            tol = 1e-13 if equal else 1e-9
            assert np.abs(np.sort(s[:N]) - ev).max() <= tol * np.abs(ev).max(), (s[:N], ev)
            for p in range(N):
                z = np.array([Z[p, 3 * m + k] for m in range(M) for k in (0, 1)])
                if np.abs(z).max() == 0.0:
                    continue
                res = J @ z - s[p] * z
                assert np.abs(res).max() <= (1e-12 if equal else 1e-8) * np.abs(J).max() * np.abs(z).max()


def _layer_state(n, B, etas):
    """Layers at rest between the surfaces etas (top first) above B."""
    M = len(etas)
    q = np.zeros((3 * M, n, n))
    lower = B
    for m in range(M - 1, -1, -1):
        top = np.maximum(etas[m], lower)
        q[3 * m] = top - lower
        lower = top
    return q


SURF = {3: (0.0, -0.4, -0.8), 4: (0.0, -0.3, -0.6, -0.9)}


@pytest.mark.parametrize("M", [3, 4])
def test_multilayer_lake_at_rest(orc, M):
    n = 24
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x)
    B = -1.5 + 0.3 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)
    q = _layer_state(n, B, tuple(e + 0.0 * X for e in SURF[M]))
    mom = [3 * m + k for m in range(M) for k in (1, 2)]
    for order in (1, 2):
        P = orc.params(M=M, rho=RHO[M], dry_tol=1e-6, order=order)
        qn = q.copy()
        for _ in range(5):
            qn, _, _ = orc.step_walled(P, qn, B, 1.0 / n, 1.0 / n, 0.3 / n / 4.0)
        assert np.abs(qn[mom]).max() <= 1e-13
        assert np.abs(qn - q).max() <= 1e-13


@pytest.mark.parametrize("M", [3, 4])
def test_multilayer_mass_and_mirror_symmetry(orc, M):
    n = 30
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x)
    B = -1.5 + 0.2 * X
    eta1 = 0.03 * np.exp(-((X - 0.4) ** 2 + (Y - 0.5) ** 2) / 0.01)
    q = _layer_state(n, B, (eta1,) + tuple(e + 0.0 * X for e in SURF[M][1:]))
    P = orc.params(M=M, rho=RHO[M], dry_tol=1e-6)
    qn = q.copy()
    for _ in range(10):
        qn, _, lost = orc.step_walled(P, qn, B, 1.0 / n, 1.0 / n, 0.3 / n / 4.0)
        assert lost == 0
    for m in range(M):
        assert abs(qn[3 * m].sum() - q[3 * m].sum()) <= 1e-13 * q[3 * m].sum()
    # y mirror: flip the state and B in y, negate hv; the result flips the same way
    hv = [3 * m + 2 for m in range(M)]
    qf = q[:, ::-1, :].copy()
    qf[hv] *= -1.0
    Bf = B[::-1, :].copy()
    qfn = qf.copy()
    for _ in range(10):
        qfn, _, _ = orc.step_walled(P, qfn, Bf, 1.0 / n, 1.0 / n, 0.3 / n / 4.0)
    back = qfn[:, ::-1, :].copy()
    back[hv] *= -1.0
    assert np.abs(back - qn).max() <= 1e-13 * np.abs(qn).max()
