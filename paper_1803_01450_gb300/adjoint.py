"""Gauge-misfit gradients through the hand-written adjoint, as a torch.autograd.Function.

The loss is J = sum over steps n = 1..N and gauges g of (eta_1(cell_g, Q^n) - obs[n-1, g])^2
for N first-order, fixed-dt steps of the two-layer model on one walled grid. The controls
are the initial surface eta_1 and the bathymetry B; the fluid starts at rest with the
interface at eta_2 (Sec. 2.1, Eqs. (4)-(5)). The map from the controls to the initial
state, the forward pass, the checkpointed backward pass and the chain rule back to the
controls all run in the CUDA library (mlswe_fixed_forward / mlswe_fixed_backward); this
module moves device pointers and nothing else.
"""
from __future__ import annotations

import numpy as np

import paper_1803_01450_gb300 as _pkg


def _device_tensor(x, device):
    """x as a contiguous float64 CUDA tensor (numpy arrays are uploaded once)."""
    import torch
    if isinstance(x, torch.Tensor):
        return x.detach().to(device=device, dtype=torch.float64).contiguous()
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device=device)


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
        self._ready = False

    def forward(self, eta1, B, device=None) -> float:
        """J for the controls eta1, B ([ny, nx] numpy arrays or CUDA tensors)."""
        import torch
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        e, b = _device_tensor(eta1, dev), _device_tensor(B, dev)
        torch.cuda.current_stream(dev).synchronize()  # the library works on its own stream
        if not self._ready:
            # the adjoint's tile timing runs on the problem's own initial state
            self.H.fixed_set_controls(e.data_ptr(), b.data_ptr(), self.eta2)
            self.H.set_dt(0, self.dt)
            self.H.adjoint_setup(self.n_steps, self.ckpt_every, self.gauge_ij, self.obs)
            self._ready = True
        return self.H.fixed_forward(e.data_ptr(), b.data_ptr(), self.eta2)

    def control_gradient(self, device):
        """(dJ/d eta_1(0), dJ/dB) of the last forward pass, [ny, nx] CUDA tensors."""
        import torch
        d_eta1 = torch.empty((self.ny, self.nx), dtype=torch.float64, device=device)
        d_B = torch.empty((self.ny, self.nx), dtype=torch.float64, device=device)
        torch.cuda.current_stream(device).synchronize()
        self.H.fixed_backward(d_eta1.data_ptr(), d_B.data_ptr())
        return d_eta1, d_B

    def backward(self, device):
        """(dJ/dQ^0 [6, ny, nx], dJ/dB at fixed Q^0 [ny, nx]) of the last forward pass."""
        import torch
        dq0 = torch.empty((6, self.ny, self.nx), dtype=torch.float64, device=device)
        dB = torch.empty((self.ny, self.nx), dtype=torch.float64, device=device)
        torch.cuda.current_stream(device).synchronize()
        self.H.fixed_backward_state(dq0.data_ptr(), dB.data_ptr())
        return dq0, dB

    def close(self):
        self.H.close()


def _make_function():
    import torch

    class GaugeMisfit(torch.autograd.Function):
        """loss = GaugeMisfit.apply(eta1_0, B, problem); eta1_0, B: float64 CUDA tensors [ny, nx]."""

        @staticmethod
        def forward(ctx, eta1_0, B, problem):
            loss = problem.forward(eta1_0, B, eta1_0.device)
            ctx.problem = problem
            ctx.device = eta1_0.device
            return torch.tensor(loss, dtype=torch.float64, device=eta1_0.device)

        @staticmethod
        def backward(ctx, g):
            d_eta1, d_B = ctx.problem.control_gradient(ctx.device)
            return g * d_eta1, g * d_B, None

    return GaugeMisfit


_GM = None


def gauge_misfit(eta1_0, B, problem: FixedGridProblem):
    """Differentiable gauge misfit of the fixed-grid problem (see module docstring)."""
    global _GM
    if _GM is None:
        _GM = _make_function()
    return _GM.apply(eta1_0, B, problem)
