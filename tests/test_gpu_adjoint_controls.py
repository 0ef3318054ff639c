"""The adjoint's control interface (the C ABI's mlswe_fixed_forward / mlswe_fixed_backward):
the initial state is built from eta_1(0) and B on the device (fluid at rest, interface at
eta_2, Sec. 2.1 Eqs. (4)-(5)), and the gradient comes back with respect to those controls.
Checked against the oracle's discrete adjoint mapped through the same control map by hand:
dJ/d eta_1 = dJ/dh_1(0), dJ/dB = dJ/dB|_Q0 - dJ/dh_2(0)."""
import numpy as np
import pytest

import oracle as O
from oracle import adjoint as OA
from paper_1803_01450_gb300 import inputs as I

pytestmark = pytest.mark.gpu
EINVAL = 1


def _setup(n=40, steps=10, n_g=8, seed=5):
    L = 1e5
    B = I.adjoint_bathymetry(n, L)
    eta1 = I.adjoint_eta1(n, seed=4000 + seed, L=L)
    gauges = I.gauge_cells(n, n_g, seed=4100 + seed)
    dx = L / n
    dt = 0.5 * dx / 205.0
    P = O.params(M=2, dry_tol=1e-3, order=1)
    truth = OA.initial_state(I.adjoint_eta1(n, seed=4001 + seed, L=L), B)
    _, states = OA.forward(P, truth, B, dx, dx, dt, steps, gauges, np.zeros((steps, n_g)))
    obs = np.stack([OA.eta1(states[k + 1], B)[gauges[:, 1], gauges[:, 0]] for k in range(steps)])
    return dict(n=n, L=L, B=B, eta1=eta1, gauges=gauges, dx=dx, dt=dt, P=P, steps=steps, obs=obs)


def test_control_gradient_matches_oracle_chain_rule(mlswe_lib):
    import torch
    from paper_1803_01450_gb300.adjoint import FixedGridProblem, gauge_misfit
    s = _setup()
    dev = torch.device("cuda", 0)
    prob = FixedGridProblem(s["n"], s["n"], s["L"], s["dt"], s["steps"], 4, s["gauges"], s["obs"])
    e = torch.tensor(s["eta1"], dtype=torch.float64, device=dev, requires_grad=True)
    b = torch.tensor(s["B"], dtype=torch.float64, device=dev, requires_grad=True)
    loss = gauge_misfit(e, b, prob)
    loss.backward()
    q0 = OA.initial_state(s["eta1"], s["B"])
    Jo, dq0o, dBo = OA.gradient(s["P"], q0, s["B"], s["dx"], s["dx"], s["dt"], s["steps"], s["gauges"], s["obs"])
    assert abs(float(loss.detach()) - Jo) <= 1e-12 * Jo
    ge, gB = e.grad.cpu().numpy(), b.grad.cpu().numpy()
    want_e, want_B = dq0o[0], dBo - dq0o[3]
    assert np.abs(ge - want_e).max() <= 1e-11 * np.abs(want_e).max()
    assert np.abs(gB - want_B).max() <= 1e-11 * np.abs(want_B).max()
    # the device-built initial state is the oracle's (one subtraction per depth, exactly)
    prob.H.fixed_set_controls(e.detach().data_ptr(), b.detach().data_ptr(), prob.eta2)
    assert np.array_equal(prob.H.get_state(0, 0), q0)
    prob.close()


def test_host_pointers_are_rejected_before_any_launch(mlswe_lib):
    """Controls and gradient outputs must be device memory; host arrays return EINVAL."""
    s = _setup(n=16, steps=2, n_g=2)
    cfg = mlswe_lib.Config(M=2, dry_tol=1e-3, order=1, max_levels=1)
    H = mlswe_lib.Hierarchy(cfg, [(0.0, 0.0, s["L"], s["L"], 16, 16)])
    eta1 = np.ascontiguousarray(s["eta1"])
    B = np.ascontiguousarray(s["B"])
    for fn in (lambda: H.fixed_set_controls(eta1.ctypes.data, B.ctypes.data, -200.0),
               lambda: H.fixed_forward(eta1.ctypes.data, B.ctypes.data, -200.0)):
        with pytest.raises(mlswe_lib.MLSWEError) as ei:
            fn()
        assert ei.value.status == EINVAL
    H.close()
