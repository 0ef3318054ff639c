"""GPU discrete adjoint (hand-written transposed sweeps, checkpointed backward pass) against
the oracle's dual-number adjoint and against central finite differences of the GPU forward
loss; the torch.autograd.Function wrapper; checkpoint spacing does not change the result."""
import numpy as np
import pytest

import oracle as O
from oracle import adjoint as OA
from paper_1803_01450_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _setup(n=48, steps=12, n_g=8, seed=3):
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


def _gpu_grad(pkg, s, ckpt):
    import torch
    from paper_1803_01450_gb300.adjoint import FixedGridProblem
    prob = FixedGridProblem(s["n"], s["n"], s["L"], s["dt"], s["steps"], ckpt, s["gauges"], s["obs"])
    J = prob.forward(s["eta1"], s["B"])
    dq0, dB = prob.backward(torch.device("cuda", 0))
    out = (J, dq0.cpu().numpy(), dB.cpu().numpy())
    prob.close()
    return out


def test_gradient_matches_oracle_adjoint(mlswe_lib):
    s = _setup()
    J, dq0, dB = _gpu_grad(mlswe_lib, s, ckpt=5)
    q0 = OA.initial_state(s["eta1"], s["B"])
    Jo, dq0o, dBo = OA.gradient(s["P"], q0, s["B"], s["dx"], s["dx"], s["dt"], s["steps"], s["gauges"], s["obs"])
    assert abs(J - Jo) <= 1e-12 * Jo
    for f in range(6):
        sc = max(np.abs(dq0o[f]).max(), 1e-300)
        assert np.abs(dq0[f] - dq0o[f]).max() <= 1e-10 * sc, (f, np.abs(dq0[f] - dq0o[f]).max() / sc)
    assert np.abs(dB - dBo).max() <= 1e-10 * np.abs(dBo).max()


def test_checkpoint_spacing_does_not_change_gradient(mlswe_lib):
    s = _setup(n=32, steps=10)
    a = _gpu_grad(mlswe_lib, s, ckpt=3)
    b = _gpu_grad(mlswe_lib, s, ckpt=10)
    assert a[0] == b[0]
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_gradient_matches_central_fd_of_gpu_forward(mlswe_lib):
    """Directional derivatives along seeded Gaussian directions mixing both controls."""
    import torch
    from paper_1803_01450_gb300.adjoint import FixedGridProblem, gauge_misfit
    s = _setup(n=64, steps=20, n_g=16)
    prob = FixedGridProblem(s["n"], s["n"], s["L"], s["dt"], s["steps"], 20, s["gauges"], s["obs"])
    dev = torch.device("cuda", 0)
    e = torch.tensor(s["eta1"], dtype=torch.float64, device=dev, requires_grad=True)
    Bt = torch.tensor(s["B"], dtype=torch.float64, device=dev, requires_grad=True)
    loss = gauge_misfit(e, Bt, prob)
    loss.backward()
    ge, gB = e.grad.cpu().numpy(), Bt.grad.cpu().numpy()
    rng = np.random.default_rng(9)
    x_norm = np.sqrt(np.sum(s["eta1"] ** 2) + np.sum(s["B"] ** 2))
    for _ in range(8):
        de = rng.standard_normal(ge.shape)
        dB = rng.standard_normal(gB.shape)
        d_norm = np.sqrt(np.sum(de ** 2) + np.sum(dB ** 2))
        eps = 1e-6 * x_norm / d_norm
        Jp = prob.forward(s["eta1"] + eps * de, s["B"] + eps * dB)
        Jm = prob.forward(s["eta1"] - eps * de, s["B"] - eps * dB)
        fd = (Jp - Jm) / (2 * eps)
        ad = float(np.sum(ge * de) + np.sum(gB * dB))
        assert abs(fd - ad) <= 1e-6 * abs(fd), (fd, ad)
    prob.close()
