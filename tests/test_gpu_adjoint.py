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


def _gpu_grad(pkg, s, ckpt, keep_edge_data=True):
    import torch
    from paper_1803_01450_gb300.adjoint import FixedGridProblem
    prob = FixedGridProblem(s["n"], s["n"], s["L"], s["dt"], s["steps"], ckpt, s["gauges"], s["obs"],
                            keep_edge_data=keep_edge_data)
    J = prob.forward(s["eta1"], s["B"])
    dq0, dB = prob.backward(torch.device("cuda", 0))
    out = (J, dq0.cpu().numpy(), dB.cpu().numpy())
    prob.close()
    return out


@pytest.mark.parametrize("keep_edge_data", [True, False])
def test_gradient_matches_oracle_adjoint(mlswe_lib, keep_edge_data):
    """Both forms of the transposed sweep: reading the per-edge forward records the
    recomputation kept, and rebuilding them per edge."""
    s = _setup()
    J, dq0, dB = _gpu_grad(mlswe_lib, s, ckpt=5, keep_edge_data=keep_edge_data)
    q0 = OA.initial_state(s["eta1"], s["B"])
    Jo, dq0o, dBo = OA.gradient(s["P"], q0, s["B"], s["dx"], s["dx"], s["dt"], s["steps"], s["gauges"], s["obs"])
    assert abs(J - Jo) <= 1e-12 * Jo
    for f in range(6):
        sc = max(np.abs(dq0o[f]).max(), 1e-300)
        assert np.abs(dq0[f] - dq0o[f]).max() <= 1e-11 * sc, (f, np.abs(dq0[f] - dq0o[f]).max() / sc)
    assert np.abs(dB - dBo).max() <= 1e-11 * np.abs(dBo).max()


def test_gradient_dot_product_with_oracle_tangent(mlswe_lib):
    """<GPU gradient, v> equals the oracle's forward-mode (dual-number) directional
    derivative of the loss along v, for random directions through every state field and
    the bathymetry."""
    s = _setup()
    J, dq0, dB = _gpu_grad(mlswe_lib, s, ckpt=5)
    q0 = OA.initial_state(s["eta1"], s["B"])
    rng = np.random.default_rng(11)
    scale = np.array([1e-2, 1.0, 1.0, 1e-2, 1.0, 1.0])[:, None, None]
    for _ in range(4):
        vq = rng.standard_normal(q0.shape) * scale
        vB = 1e-2 * rng.standard_normal(s["B"].shape)
        Jt, dJ = OA.tangent(s["P"], q0, s["B"], s["dx"], s["dx"], s["dt"], s["steps"], s["gauges"], s["obs"], vq, vB)
        assert abs(Jt - J) <= 1e-12 * Jt
        ad = float(np.sum(dq0 * vq) + np.sum(dB * vB))
        assert abs(ad - dJ) <= 1e-11 * abs(dJ), (ad, dJ)


def test_kept_and_rebuilt_edge_records_agree(mlswe_lib):
    """The two forms differ only in where the forward quantities are computed (the sweep
    kernel's arithmetic or the VJP's), so the gradients agree to rounding."""
    s = _setup(n=40, steps=8)
    a = _gpu_grad(mlswe_lib, s, ckpt=4, keep_edge_data=True)
    b = _gpu_grad(mlswe_lib, s, ckpt=4, keep_edge_data=False)
    assert a[0] == b[0]  # the forward pass is the same
    for f in range(6):
        sc = max(np.abs(b[1][f]).max(), 1e-300)
        assert np.abs(a[1][f] - b[1][f]).max() <= 1e-12 * sc
    assert np.abs(a[2] - b[2]).max() <= 1e-12 * np.abs(b[2]).max()


def test_checkpoint_spacing_does_not_change_gradient(mlswe_lib):
    s = _setup(n=32, steps=10)
    a = _gpu_grad(mlswe_lib, s, ckpt=3)
    b = _gpu_grad(mlswe_lib, s, ckpt=10)
    assert a[0] == b[0]
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_gradient_matches_central_fd_of_gpu_forward(mlswe_lib):
    """Directional derivatives along 64 seeded Gaussian directions mixing both controls."""
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
    for _ in range(64):
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


def test_recording_sweep_reproduces_plain_steps(mlswe_lib):
    """With the per-edge records kept, the forward pass steps its last segment with the
    recording form of the sweep kernel; its state must equal plain level steps bit for bit
    (the recorded steps are the ones the backward pass differentiates)."""
    s = _setup(n=32, steps=6)
    from paper_1803_01450_gb300.adjoint import FixedGridProblem
    prob = FixedGridProblem(s["n"], s["n"], s["L"], s["dt"], s["steps"], s["steps"], s["gauges"], s["obs"],
                            keep_edge_data=True)
    prob.forward(s["eta1"], s["B"])
    q_rec = prob.H.get_state(0, 0)
    prob.close()
    cfg = mlswe_lib.Config(M=2, dry_tol=1e-3, order=1, max_levels=1)
    H = mlswe_lib.Hierarchy(cfg, [(0.0, 0.0, s["L"], s["L"], s["n"], s["n"])])
    H.set_bathymetry(0, s["B"])
    H.set_state(0, 0, OA.initial_state(s["eta1"], s["B"]))
    H.set_dt(0, s["dt"])
    for _ in range(s["steps"]):
        H.step_level(0)
    assert np.array_equal(H.get_state(0, 0), q_rec)
    H.close()


def test_full_size_gradient(mlswe_lib):
    """The adjoint workload at full size (512^2, 200 first-order steps, 32 gauges), as the
    bench runs it: checkpoints every 20 steps and one segment give the same gradient bit for
    bit, and directional derivatives along 4 seeded directions match central differences of
    the GPU forward loss."""
    import torch
    from paper_1803_01450_gb300.adjoint import FixedGridProblem, gauge_misfit
    n, L, steps, n_g = 512, 1e5, 200, 32
    B = I.adjoint_bathymetry(n, L)
    eta1 = I.adjoint_eta1(n, seed=4000, L=L)
    gauges = I.gauge_cells(n, n_g, seed=4100)
    dt = 0.5 * (L / n) / 205.0
    obs = np.zeros((steps, n_g))
    dev = torch.device("cuda", 0)
    grads = []
    for ckpt in (20, 200):
        prob = FixedGridProblem(n, n, L, dt, steps, ckpt, gauges, obs)
        e = torch.tensor(eta1, dtype=torch.float64, device=dev, requires_grad=True)
        Bt = torch.tensor(B, dtype=torch.float64, device=dev, requires_grad=True)
        loss = gauge_misfit(e, Bt, prob)
        loss.backward()
        grads.append((float(loss.detach()), e.grad.cpu().numpy(), Bt.grad.cpu().numpy()))
        if ckpt == 20:
            keep = prob
        else:
            prob.close()
    assert grads[0][0] == grads[1][0]
    assert np.array_equal(grads[0][1], grads[1][1]) and np.array_equal(grads[0][2], grads[1][2])
    _, ge, gB = grads[0]
    rng = np.random.default_rng(19)
    x_norm = np.sqrt(np.sum(eta1 ** 2) + np.sum(B ** 2))
    for _ in range(4):
        de = rng.standard_normal(ge.shape)
        dB = rng.standard_normal(gB.shape)
        d_norm = np.sqrt(np.sum(de ** 2) + np.sum(dB ** 2))
        eps = 1e-6 * x_norm / d_norm
        Jp = keep.forward(eta1 + eps * de, B + eps * dB)
        Jm = keep.forward(eta1 - eps * de, B - eps * dB)
        fd = (Jp - Jm) / (2 * eps)
        ad = float(np.sum(ge * de) + np.sum(gB * dB))
        assert abs(fd - ad) <= 1e-6 * abs(fd), (fd, ad)
    keep.close()
