"""Oracle of the gauge-misfit gradient (discrete adjoint of the fixed-grid, first-order step).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

J = sum_{n=1..N} sum_g (eta_1(cell_g, Q^n) - obs[n-1, g])^2, eta_1 = B + h_2 + h_1 (Eq. (4)).
The gradient is the plain definition of the adjoint: every state of the forward run is
kept (no checkpointing), and the transposed Jacobian of each step is applied in reverse,
with the step Jacobian taken exactly by the oracle's forward-mode dual numbers
(or_adjoint_step). The initial state is parameterised by the controls as
h_2 = eta_2 - B, h_1 = eta_1 - eta_2, momenta 0.
"""
from __future__ import annotations

import numpy as np

import oracle as O


def eta1(q, B):
    return B + q[3] + q[0]


def initial_state(eta1_0, B, eta2=-200.0):
    z = np.zeros_like(B)
    return np.stack([eta1_0 - eta2, z, z.copy(), eta2 - B, z.copy(), z.copy()])


def forward(P, q0, B, dx, dy, dt, n_steps, gauge_ij, obs, keep=True):
    gi, gj = gauge_ij[:, 0], gauge_ij[:, 1]
    q = q0.copy()
    states = [q.copy()] if keep else None
    J = 0.0
    for n in range(1, n_steps + 1):
        q, _, _ = O.step_walled(P, q, B, dx, dy, dt)
        r = eta1(q, B)[gj, gi] - obs[n - 1]
        J += float(np.sum(r * r))
        if keep:
            states.append(q.copy())
    return J, states


def gradient(P, q0, B, dx, dy, dt, n_steps, gauge_ij, obs):
    """(J, dJ/dQ^0 [6][ny][nx], dJ/dB [ny][nx]) with B entering steps and gauges."""
    J, states = forward(P, q0, B, dx, dy, dt, n_steps, gauge_ij, obs)
    gi, gj = gauge_ij[:, 0], gauge_ij[:, 1]
    lam = np.zeros_like(q0)
    gB = np.zeros_like(B)
    for n in range(n_steps - 1, -1, -1):
        qn1 = states[n + 1]
        r = eta1(qn1, B)[gj, gi] - obs[n]
        for k, (i, j) in enumerate(zip(gi, gj)):
            lam[0, j, i] += 2.0 * r[k]
            lam[3, j, i] += 2.0 * r[k]
            gB[j, i] += 2.0 * r[k]
        lam, gBs = O.adjoint_step(P, states[n], B, dx, dy, dt, lam)
        gB += gBs
    return J, lam, gB


def control_gradient(P, eta1_0, B, dx, dy, dt, n_steps, gauge_ij, obs, eta2=-200.0):
    """(J, dJ/d eta1_0, dJ/dB) for the controls (the rest-state parameterisation)."""
    q0 = initial_state(eta1_0, B, eta2)
    J, dq0, gB = gradient(P, q0, B, dx, dy, dt, n_steps, gauge_ij, obs)
    return J, dq0[0], gB - dq0[3]


def tangent(P, q0, B, dx, dy, dt, n_steps, gauge_ij, obs, dq0, dB):
    """(J, dJ along (dq0, dB)) by forward-mode dual numbers through every step
    (or_tangent_loss): the exact directional derivative the adjoint's gradient must match
    in a dot product."""
    import ctypes
    q0 = np.ascontiguousarray(q0, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    dq0 = np.ascontiguousarray(dq0, dtype=np.float64)
    dB = np.ascontiguousarray(dB, dtype=np.float64)
    g = np.ascontiguousarray(np.asarray(gauge_ij, dtype=np.int32).reshape(-1, 2))
    o = np.ascontiguousarray(np.asarray(obs, dtype=np.float64).reshape(n_steps, len(g)))
    ny, nx = B.shape
    J = ctypes.c_double(0.0)
    dJ = ctypes.c_double(0.0)
    dp = ctypes.POINTER(ctypes.c_double)
    O.lib().or_tangent_loss(ctypes.byref(P), nx, ny, ctypes.c_double(dx), ctypes.c_double(dy), ctypes.c_double(dt),
                            n_steps, q0.ctypes.data_as(dp), B.ctypes.data_as(dp), dq0.ctypes.data_as(dp),
                            dB.ctypes.data_as(dp), len(g), g.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                            o.ctypes.data_as(dp), ctypes.byref(J), ctypes.byref(dJ))
    return J.value, dJ.value
