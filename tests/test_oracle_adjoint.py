"""Pins of the oracle's discrete adjoint: against central finite differences of the
oracle's own forward loss (which uses no derivative code at all), per step and for the
whole gauge-misfit problem, for both controls."""
import numpy as np
import pytest

import oracle as O
from oracle import adjoint as A
from paper_1803_01450_gb300 import inputs as I


def _problem(n=20, steps=6, n_g=5, seed=0):
    L = 1e5
    x = I.centers(0.0, L, n)
    X, Y = np.meshgrid(x, x)
    B = -4000.0 + 500.0 * np.sin(2 * np.pi * X / L) * np.cos(2 * np.pi * Y / L)
    rng = np.random.default_rng(seed)
    eta1 = 0.0
    for _ in range(2):
        eta1 = eta1 + rng.uniform(0.5, 2.0) * np.exp(-((X - rng.uniform(2e4, 8e4)) ** 2 +
                                                     (Y - rng.uniform(2e4, 8e4)) ** 2) / 1.5e4 ** 2)
    gauges = np.stack([rng.integers(1, n - 1, n_g), rng.integers(1, n - 1, n_g)], axis=1).astype(np.int32)
    dx = L / n
    dt = 0.5 * dx / 205.0
    P = O.params(M=2, dry_tol=1e-3, order=1)
    # observations: a run from a slightly different initial surface
    q_true = A.initial_state(1.1 * eta1, B)
    _, states = A.forward(P, q_true, B, dx, dx, dt, steps, gauges, np.zeros((steps, n_g)))
    obs = np.stack([A.eta1(states[k + 1], B)[gauges[:, 1], gauges[:, 0]] for k in range(steps)])
    return P, eta1, B, dx, dt, steps, gauges, obs


def test_adjoint_step_is_transpose_of_step():
    """<lam, (Q(q + e d) - Q(q - e d)) / 2e> = <adjoint(lam), d> for random d, lam."""
    P, eta1, B, dx, dt, _, _, _ = _problem(n=16)
    q = A.initial_state(eta1, B)
    rng = np.random.default_rng(1)
    q[1] = 0.3 * rng.standard_normal(q[1].shape) * q[0] / 200.0
    q[5] = 0.3 * rng.standard_normal(q[5].shape) * q[3] / 3000.0
    for _ in range(3):
        d = rng.standard_normal(q.shape) * np.array([1e-2, 1e-1, 1e-1, 1e-2, 1e-1, 1e-1])[:, None, None]
        lam = rng.standard_normal(q.shape)
        eps = 1e-3
        qp, _, _ = O.step_walled(P, q + eps * d, B, dx, dx, dt)
        qm, _, _ = O.step_walled(P, q - eps * d, B, dx, dx, dt)
        lhs = np.sum(lam * (qp - qm)) / (2 * eps)
        lam_n, gB = O.adjoint_step(P, q, B, dx, dx, dt, lam)
        rhs = np.sum(lam_n * d)
        assert abs(lhs - rhs) <= 1e-7 * max(abs(lhs), abs(rhs), 1e-30), (lhs, rhs)
        # bathymetry direction
        dB = rng.standard_normal(B.shape)
        qp, _, _ = O.step_walled(P, q, B + eps * dB, dx, dx, dt)
        qm, _, _ = O.step_walled(P, q, B - eps * dB, dx, dx, dt)
        lhs = np.sum(lam * (qp - qm)) / (2 * eps)
        rhs = np.sum(gB * dB)
        assert abs(lhs - rhs) <= 1e-7 * max(abs(lhs), abs(rhs), 1e-30), (lhs, rhs)


def test_gauge_misfit_gradient_matches_central_fd():
    P, eta1, B, dx, dt, steps, gauges, obs = _problem()
    J, g_eta, g_B = A.control_gradient(P, eta1, B, dx, dx, dt, steps, gauges, obs)
    assert J > 0
    rng = np.random.default_rng(2)
    for _ in range(4):
        de = rng.standard_normal(eta1.shape)
        dB = rng.standard_normal(B.shape)
        eps = 1e-4
        Jp, _ = A.forward(P, A.initial_state(eta1 + eps * de, B + eps * dB), B + eps * dB, dx, dx, dt, steps, gauges,
                          obs, keep=False)
        Jm, _ = A.forward(P, A.initial_state(eta1 - eps * de, B - eps * dB), B - eps * dB, dx, dx, dt, steps, gauges,
                          obs, keep=False)
        fd = (Jp - Jm) / (2 * eps)
        ad = float(np.sum(g_eta * de) + np.sum(g_B * dB))
        assert abs(fd - ad) <= 1e-6 * abs(fd), (fd, ad)


def test_adjoint_dot_product_with_dual_number_tangent():
    """<gradient, v> of the reverse-mode adjoint equals the forward-mode (dual-number)
    directional derivative of the same loss along v, for random directions through every
    state field and the bathymetry: two exact derivatives, independent code, equal to
    rounding."""
    P, eta1, B, dx, dt, steps, gauges, obs = _problem()
    q0 = A.initial_state(eta1, B)
    rng = np.random.default_rng(7)
    q0[1] = 0.2 * rng.standard_normal(q0[1].shape) * q0[0] / 200.0  # some motion in both layers
    q0[5] = 0.2 * rng.standard_normal(q0[5].shape) * q0[3] / 3000.0
    J, dq0, gB = A.gradient(P, q0, B, dx, dx, dt, steps, gauges, obs)
    scale = np.array([1e-2, 1.0, 1.0, 1e-2, 1.0, 1.0])[:, None, None]
    for _ in range(4):
        vq = rng.standard_normal(q0.shape) * scale
        vB = 1e-2 * rng.standard_normal(B.shape)
        Jt, dJ = A.tangent(P, q0, B, dx, dx, dt, steps, gauges, obs, vq, vB)
        assert abs(Jt - J) <= 1e-14 * J
        ad = float(np.sum(dq0 * vq) + np.sum(gB * vB))
        assert abs(ad - dJ) <= 1e-13 * abs(dJ), (ad, dJ, abs(ad - dJ) / abs(dJ))
