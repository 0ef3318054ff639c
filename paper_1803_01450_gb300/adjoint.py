"""Gauge-misfit gradients through the hand-written adjoint, as a torch.autograd.Function.

The loss is J = sum over steps n = 1..N and gauges g of (eta_1(cell_g, Q^n) - obs[n-1, g])^2
for N first-order, fixed-dt steps of the two-layer model on one walled grid. The controls
are the initial surface eta_1 (the fluid starts at rest, the interface at eta_2) and the
bathymetry B:
    h_2 = eta_2 - B,   h_1 = eta_1 - eta_2,   momenta 0,
so dJ/d eta_1 = dJ/dh_1(0) and dJ/dB = (dJ/dB through the steps and gauges) - dJ/dh_2(0).
Forward, backward (with checkpointing) and the transposed steps all run in the CUDA
library; this module only maps the controls to the initial state and back.
"""
from __future__ import annotations

import numpy as np

import paper_1803_01450_gb300 as _pkg


class FixedGridProblem:
    """One walled grid, a fixed time step, gauges and observations."""

    def __init__(self, nx, ny, L, dt, n_steps, ckpt_every, gauge_ij, obs, eta2=-200.0, dry_tol=1e-3,
                 stream=None, keep_edge_data=True):
        self.nx, self.ny, self.L, self.dt = nx, ny, L, dt
        self.n_steps, self.ckpt_every = n_steps, ckpt_every
        self.gauge_ij = np.asarray(gauge_ij, dtype=np.int32)
        self.obs = np.asarray(obs, dtype=np.float64)
        self.eta2 = eta2
        cfg = _pkg.Config(M=2, dry_tol=dry_tol, order=1, max_levels=1)
        self.H = _pkg.Hierarchy(cfg, [(0.0, 0.0, L, L, nx, ny)], stream=stream)
        self.H.adjoint_keep_edge_data(keep_edge_data)

    def initial_state(self, eta1, B):
        h2 = self.eta2 - B
        h1 = eta1 - self.eta2
        z = np.zeros_like(B)
        return np.stack([h1, z, z, h2, z.copy(), z.copy()])

    def forward(self, eta1: np.ndarray, B: np.ndarray) -> float:
        self.H.set_bathymetry(0, B)
        self.H.set_state(0, 0, self.initial_state(eta1, B))
        self.H.set_dt(0, self.dt)
        self.H.adjoint_setup(self.n_steps, self.ckpt_every, self.gauge_ij, self.obs)
        return self.H.fixed_forward()

    def backward(self, device):
        import torch
        dq0 = torch.empty((6, self.ny, self.nx), dtype=torch.float64, device=device)
        dB = torch.empty((self.ny, self.nx), dtype=torch.float64, device=device)
        torch.cuda.synchronize(device)
        self.H.fixed_backward(dq0.data_ptr(), dB.data_ptr())
        return dq0, dB

    def close(self):
        self.H.close()


def _make_function():
    import torch

    class GaugeMisfit(torch.autograd.Function):
        """loss = GaugeMisfit.apply(eta1_0, B, problem); eta1_0, B: float64 CUDA tensors [ny, nx]."""

        @staticmethod
        def forward(ctx, eta1_0, B, problem):
            loss = problem.forward(eta1_0.detach().cpu().numpy(), B.detach().cpu().numpy())
            ctx.problem = problem
            ctx.device = eta1_0.device
            return torch.tensor(loss, dtype=torch.float64, device=eta1_0.device)

        @staticmethod
        def backward(ctx, g):
            dq0, dB = ctx.problem.backward(ctx.device)
            d_eta1 = dq0[0]
            d_B = dB - dq0[3]
            return g * d_eta1, g * d_B, None

    return GaugeMisfit


_GM = None


def gauge_misfit(eta1_0, B, problem: FixedGridProblem):
    """Differentiable gauge misfit of the fixed-grid problem (see module docstring)."""
    global _GM
    if _GM is None:
        _GM = _make_function()
    return _GM.apply(eta1_0, B, problem)
