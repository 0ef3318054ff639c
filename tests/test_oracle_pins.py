"""Pins of the FP64 oracle's solver step against facts fixed outside the oracle.

Each test checks the oracle against something other than itself: closed forms
(eigenvalues of the two-layer system at equal velocities, the exact dam-break
solution), library routines (numpy eigenvalues of the coupled Jacobian), the
textbook Roe decomposition of dQ (a different formula from the f-wave split of
the flux jump), and invariants of the continuous problem (lake at rest, mass
conservation, mirror symmetry, reduction of two layers to one).
"""
import numpy as np
import pytest
from scipy.optimize import brentq

from paper_1803_01450_gb300 import inputs as I

G = 9.81


# --------------------------------------------------------------------- invariants
@pytest.mark.parametrize("M", [1, 2])
@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("kind", ["flat", "shelf", "shore"])
def test_lake_at_rest(orc, M, order, kind):
    """Sec. 2.1, Eqs. (3)-(4): a fluid at rest with flat surfaces stays at rest (to rounding
    of eta - B, 1e-13 of the depth scale), also where the lower layer or both layers end on
    a shore."""
    n = 48
    if kind == "flat":
        B = -4000.0 * np.ones((n, n))
    elif kind == "shelf":
        B = I.shelf_B(np.meshgrid(I.centers(0, 1e5, n), I.centers(0, 1e5, n))[0])
    else:
        B = I.shore_bathymetry(n, n)
    if M == 2:
        q = I.layered_state(B, np.zeros_like(B), -200.0 * np.ones_like(B))
    else:
        q = I.layered_state(B, np.zeros_like(B), B - 1.0)[:3]  # one layer: eta_2 below ground
    P = orc.params(M=M, order=order, dry_tol=1e-3)
    dx = 1e5 / n
    qq = q.copy()
    for _ in range(10):
        qq, _, _ = orc.step_walled(P, qq, B, dx, dx, 0.5 * dx / 210.0)
    eta0 = B + sum(q[3 * m] for m in range(M))
    eta = B + sum(qq[3 * m] for m in range(M))
    wet = q[0] > 1e-3
    assert np.abs(eta - eta0)[wet].max() <= 1e-13 * 4000
    mom = [3 * m + k for m in range(M) for k in (1, 2)]
    assert np.abs(qq[mom]).max() <= 1e-13 * 4000


@pytest.mark.parametrize("M", [1, 2])
@pytest.mark.parametrize("order", [1, 2])
def test_mass_conservation_walled(orc, M, order):
    """Mass of every layer is constant on a walled wet domain: the mass rows of the flux
    jump carry no source, so the update telescopes."""
    q, B = I.gaussian_random_state(3, M, 37, 29)
    P = orc.params(M=M, order=order, dry_tol=1e-6)
    m0 = np.array([q[3 * m].sum() for m in range(M)])
    qq = q.copy()
    for _ in range(15):
        qq, _, _ = orc.step_walled(P, qq, B, 1 / 37, 1 / 29, 0.05 / 37)
    m1 = np.array([qq[3 * m].sum() for m in range(M)])
    assert np.all(np.abs(m1 - m0) <= 1e-13 * m0)


def test_mirror_symmetry(orc):
    """The small workload (hump centred at y = 0.5 on [0,1]^2 with walls) stays symmetric
    under y -> 1 - y with hv -> -hv."""
    w = I.small(50)
    P = orc.params(M=2, dry_tol=w["dry_tol"])
    q = w["q"].copy()
    for _ in range(40):
        q, _, _ = orc.step_walled(P, q, w["B"], w["dx"], w["dy"], 0.9 * w["dx"] / 3.2)
    for f in range(6):
        ref = -q[f][::-1] if f % 3 == 2 else q[f][::-1]
        scale = max(np.abs(q[f]).max(), 1e-300)
        assert np.abs(q[f] - ref).max() <= 1e-12 * scale


def test_two_layers_with_absent_lower_layer_equal_one_layer(orc):
    """A two-layer state with h_2 = 0 everywhere evolves like the one-layer model."""
    q1, B = I.gaussian_random_state(8, 1, 30, 26)
    q2 = np.zeros((6,) + q1.shape[1:])
    q2[:3] = q1
    P1 = orc.params(M=1, dry_tol=1e-6)
    P2 = orc.params(M=2, dry_tol=1e-6)
    a, b = q1.copy(), q2.copy()
    for _ in range(10):
        a, _, _ = orc.step_walled(P1, a, B, 1 / 30, 1 / 26, 0.05 / 30)
        b, _, _ = orc.step_walled(P2, b, B, 1 / 30, 1 / 26, 0.05 / 30)
    for f in range(3):
        assert np.abs(a[f] - b[f]).max() <= 1e-13 * max(np.abs(a[f]).max(), 1e-300)
    assert np.abs(b[3:]).max() == 0.0


# ----------------------------------------------------------------- edge solver
def _roe_textbook(hL, huL, hvL, hR, huR, hvR):
    """Roe's approximate Riemann solver for the one-layer SWE on a flat bottom in its
    textbook form: eigen-decomposition of dQ (not of the flux jump) at the Roe state."""
    sL, sR = np.sqrt(hL), np.sqrt(hR)
    uL, uR, vL, vR = huL / hL, huR / hR, hvL / hL, hvR / hR
    u = (sL * uL + sR * uR) / (sL + sR)
    v = (sL * vL + sR * vR) / (sL + sR)
    c = np.sqrt(G * 0.5 * (hL + hR))
    dq = np.array([hR - hL, huR - huL, hvR - hvL])
    R = np.array([[1.0, 0.0, 1.0], [u - c, 0.0, u + c], [v, 1.0, v]])
    a = np.linalg.solve(R, dq)
    lam = np.array([u - c, u, u + c])
    am = sum(min(lam[p], 0.0) * a[p] * R[:, p] for p in range(3))
    ap = sum(max(lam[p], 0.0) * a[p] * R[:, p] for p in range(3))
    return am, ap


def test_one_layer_flat_bottom_equals_roe(orc):
    """On a flat bottom the f-wave split of the flux jump equals Roe's split of dQ (the Roe
    matrix maps dQ to df exactly for the SWE), so the fluctuations must coincide."""
    P = orc.params(M=1, dry_tol=1e-6)
    rng = np.random.default_rng(0)
    for _ in range(200):
        hL, hR = rng.uniform(0.5, 2.0, 2)
        uL, uR, vL, vR = rng.uniform(-0.8, 0.8, 4)
        qL = [hL, hL * uL, hL * vL]
        qR = [hR, hR * uR, hR * vR]
        _, s, am, ap, _ = orc.riemann(P, qL, qR, 0.0, 0.0)
        ram, rap = _roe_textbook(*qL, *qR)
        # Transverse momentum: the f-wave carries it with the Roe-averaged v (see oracle).
        assert np.allclose(am[:3], ram, rtol=1e-12, atol=1e-12)
        assert np.allclose(ap[:3], rap, rtol=1e-12, atol=1e-12)


def _two_layer_jacobian(u1, u2, h1, h2, r):
    c1, c2 = G * h1, G * h2
    return np.array([[0, 1, 0, 0], [c1 - u1 ** 2, 2 * u1, c1, 0], [0, 0, 0, 1], [r * c2, 0, c2 - u2 ** 2, 2 * u2]])


def test_eigenvalues_closed_form_at_equal_velocities(orc):
    """At u_1 = u_2 the eigenvalues of the two-layer system are u -+ sqrt(mu_+-); the guesses
    are exact there and agree with numpy's eigenvalues of the Jacobian."""
    P = orc.params(M=2)
    for (u, h1, h2) in [(0.0, 0.6, 0.4), (0.3, 200.0, 3800.0), (-1.2, 50.0, 5.0)]:
        lam, lost = orc.eigen(P, u, u, h1, h2)
        assert lost == 0
        ref = np.sort(np.linalg.eigvals(_two_layer_jacobian(u, u, h1, h2, P.r)).real)
        assert np.allclose(lam, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


def test_eigenvalues_newton_converge(orc):
    """With u_1 != u_2, two Newton steps from the guesses land on numpy's eigenvalues to the
    accuracy quadratic convergence allows, and closer than the guesses themselves."""
    P = orc.params(M=2)
    Pg = orc.params(M=2, eigen=1)
    for (u1, u2, h1, h2) in [(0.02, -0.01, 0.6, 0.4), (0.5, 0.2, 200.0, 3800.0), (0.05, 0.0, 1.0, 1.0)]:
        lam, lost = orc.eigen(P, u1, u2, h1, h2)
        guess, _ = orc.eigen(Pg, u1, u2, h1, h2)
        assert lost == 0
        ref = np.sort(np.linalg.eigvals(_two_layer_jacobian(u1, u2, h1, h2, P.r)).real)
        e2 = np.abs(lam - ref)
        e0 = np.abs(guess - ref)
        assert np.all(e2 <= np.maximum(1e-3 * e0, 1e-12 * np.abs(ref).max()))


def test_hyperbolicity_loss_flag(orc):
    P = orc.params(M=2)
    _, lost = orc.eigen(P, 1.0, -1.0, 0.6, 0.4)  # (du)^2 = 4 > (1 - r) g (h1 + h2) = 0.24
    assert lost == 1
    _, lost = orc.eigen(P, 0.1, -0.1, 0.6, 0.4)
    assert lost == 0


def _flux_jump(qL, qR, BL, BR, r):
    """Flux jump of the two-layer model with the non-conservative layer coupling
    integrated across the edge at the mean depths (written from the PDE)."""
    def f(q):
        h1, hu1, hv1, h2, hu2, hv2 = q
        return np.array([hu1, hu1 ** 2 / h1 + 0.5 * G * h1 ** 2, hu1 * hv1 / h1,
                         hu2, hu2 ** 2 / h2 + 0.5 * G * h2 ** 2, hu2 * hv2 / h2])
    qL, qR = np.asarray(qL), np.asarray(qR)
    d = f(qR) - f(qL)
    hb1, hb2 = 0.5 * (qL[0] + qR[0]), 0.5 * (qL[3] + qR[3])
    dh1, dh2, dB = qR[0] - qL[0], qR[3] - qL[3], BR - BL
    d[1] += G * hb1 * (dh2 + dB)          # layer 1 sits on layer 2 and the ground
    d[4] += G * hb2 * (r * dh1 + dB)      # layer 2 carries the weight of layer 1
    return d


def test_coupled_waves_sum_to_flux_jump_and_are_eigenvectors(orc):
    """Coupled branch: the f-waves add up to the flux jump (with the layer coupling and
    bathymetry terms), and each acoustic wave's normal part is an eigenvector of the
    Jacobian at the Roe state with its speed as eigenvalue."""
    P = orc.params(M=2, dry_tol=1e-6)
    rng = np.random.default_rng(4)
    for _ in range(100):
        h1, h2 = rng.uniform(0.3, 1.0), rng.uniform(0.3, 1.0)
        qL = [h1, 0.05 * rng.standard_normal(), 0.05 * rng.standard_normal(),
              h2, 0.05 * rng.standard_normal(), 0.05 * rng.standard_normal()]
        qR = [h1 * (1 + 0.1 * rng.standard_normal()), 0.05 * rng.standard_normal(), 0.05 * rng.standard_normal(),
              h2 * (1 + 0.1 * rng.standard_normal()), 0.05 * rng.standard_normal(), 0.05 * rng.standard_normal()]
        BL, BR = -2.0, -2.0 + 0.05 * rng.standard_normal()
        Z, s, am, ap, info = orc.riemann(P, qL, qR, BL, BR)
        d = _flux_jump(qL, qR, BL, BR, P.r)
        assert np.allclose(Z.sum(axis=0), d, rtol=0, atol=1e-13 * np.abs(d).max() + 1e-16)
        assert np.allclose(am + ap, d, rtol=0, atol=1e-13 * np.abs(d).max() + 1e-16)
        sl = np.sqrt([qL[0], qL[3]]); sr = np.sqrt([qR[0], qR[3]])
        u = [(sl[m] * qL[3 * m + 1] / qL[3 * m] + sr[m] * qR[3 * m + 1] / qR[3 * m]) / (sl[m] + sr[m]) for m in range(2)]
        A = _two_layer_jacobian(u[0], u[1], 0.5 * (qL[0] + qR[0]), 0.5 * (qL[3] + qR[3]), P.r)
        exact = np.linalg.eigvals(A).real
        for p in range(4):
            z = Z[p][[0, 1, 3, 4]]
            res = A @ z - s[p] * z
            # The eigenvalue comes from two Newton steps: the residual is bounded by its error.
            dl = np.abs(exact - s[p]).min()
            assert np.abs(res).max() <= (8.0 * dl + 1e-12 * (np.abs(s[p]) + 1.0)) * np.abs(z).max() + 1e-15


# ---------------------------------------------------------------- exact solution
def _stoker(hl, hr, x, t):
    """Exact dam-break solution of the one-layer SWE (wet both sides, flat bottom)."""
    cl = np.sqrt(G * hl)

    def fn(hm):
        um_r = 2 * (cl - np.sqrt(G * hm))
        um_s = (hm - hr) * np.sqrt(0.5 * G * (1 / hm + 1 / hr))
        return um_r - um_s

    hm = brentq(fn, hr, hl)
    um = 2 * (cl - np.sqrt(G * hm))
    sh = hm * um / (hm - hr)
    xi = x / t
    h = np.where(xi < -cl, hl, np.where(xi < um - np.sqrt(G * hm), (2 * cl - xi) ** 2 / (9 * G),
                                          np.where(xi < sh, hm, hr)))
    return h


@pytest.mark.parametrize("order", [1, 2])
def test_dam_break_converges_to_exact(orc, order):
    """1-D dam break (h = 2 | 1): the L1 error against the exact solution falls with
    resolution, faster for the second-order scheme, and is small on the finest grid."""
    P = orc.params(M=1, dry_tol=1e-6, order=order, limiter=2)
    errs = []
    for n in (100, 200, 400):
        dx = 2.0 / n
        x = -1.0 + (np.arange(n) + 0.5) * dx
        line = np.zeros((n + 4, 3))
        line[2:-2, 0] = np.where(x < 0, 2.0, 1.0)
        Bl = np.zeros(n + 4)
        t, T = 0.0, 0.15
        dt = 0.4 * dx / (np.sqrt(G * 2.0) * 1.5)
        while t < T - 1e-14:
            step = min(dt, T - t)
            line[:2] = line[2]; line[-2:] = line[-3]  # zero-gradient ends
            out, _, _ = orc.sweep_line(P, line, Bl, step / dx)
            line[2:-2] = out
            t += step
        errs.append(np.abs(line[2:-2, 0] - _stoker(2.0, 1.0, x, T)).sum() * dx)
    assert errs[1] < 0.75 * errs[0] and errs[2] < 0.75 * errs[1], errs
    assert errs[2] < (0.01 if order == 2 else 0.02), errs
