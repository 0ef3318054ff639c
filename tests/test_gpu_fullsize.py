"""The batched-AMR workload at full size, in the launch configuration the benchmark times
(512^2 coarse, ratios 4, 4, 1000 + 3000 seeded patches over the shore bathymetry,
autotuned tiles, one persistent launch per level step, graph replay), checked where the
oracle can follow it: a level-2 step of sampled patches (the most active and some at
random) against the oracle's patch step on the same ghost-filled input, and the whole
level-0 step against the oracle's walled step; and the ensemble workload (256 members) on
sampled members and patches. Within 1e-11 of each field's level-wide scale (state_scale:
a momentum's scale is at least h_max sqrt(g h_max) of its layer). The adjoint
workload at full size: its gradient against central differences of the GPU forward."""
import numpy as np
import pytest

import oracle as O
from paper_1803_01450_gb300 import inputs as I
from conftest import report, state_scale

pytestmark = pytest.mark.gpu
TOL = 1e-11
NG = 2


@pytest.fixture(scope="module")
def amr_full(mlswe_lib):
    n0, r, L = 512, 4, 1e5
    nf = n0 * r * r
    cfg = mlswe_lib.Config(M=2, dry_tol=1e-3, max_levels=3, ratio=[r, r], regrid_interval=0, min_side=16,
                           max_side=64, flag_tol=5e-5)
    H = mlswe_lib.Hierarchy(cfg, [(0.0, 0.0, L, L, n0, n0)])
    xf = I.centers(0.0, L, nf)
    H.set_bathymetry(0, np.ascontiguousarray(np.broadcast_to(I.shore_B(xf)[None, :], (nf, nf))))
    B0 = H.get_bathymetry(0, 0)
    x0 = I.centers(0.0, L, n0)
    X, Y = np.meshgrid(x0, x0)
    eta1 = I.hump_field(X, Y, *I.humps(3000, 8))
    H.set_state(0, 0, I.layered_state(B0, eta1, -200.0 * np.ones_like(B0)))
    l1 = I.random_layout(3100, n0 * r, n0 * r, 1000, r)
    l2 = I.random_layout(3200, nf, nf, 3000, r, parents=l1, margin=2)
    H.set_patches(0, 1, l1)
    H.interp_fine(0, 0)
    H.set_patches(0, 2, l2)
    H.interp_fine(1, 0)
    for lev in range(3):
        H.autotune(lev, iters=2)
    H.advance(1)
    yield H, dict(n0=n0, r=r, L=L, nf=nf)
    H.close()


def _scale(q):
    return np.maximum(np.abs(q).max(axis=(1, 2)), 1e-300)


def _check_walled_step(P, q0, B, dx, dt, got, rng, where):
    """got against the oracle's walled step of q0, every field within 1e-11 of its scale
    (state_scale of the states before and after: momenta at least h_max sqrt(g h_max))."""
    want, _, _ = O.step_walled(P, q0, B, dx, dx, dt)
    scale = np.maximum(state_scale(want, P.M), state_scale(q0, P.M))
    err = np.abs(got - want).max(axis=(1, 2)) / scale
    report(f"walled_step_{where}", err)
    assert err.max() <= TOL, (where, err)


def test_level2_sampled_patches_match_oracle_patch_step(amr_full):
    H, w = amr_full
    nf, L = w["nf"], w["L"]
    dx = L / nf
    dt = 0.03  # Courant number about 0.5 at the deepest water on this level
    boxes = H.get_patches(0, 2)
    assert len(boxes) == 3000
    H.fill_ghosts(2, 1.0)
    q0 = H.get_state(0, 2)
    B2 = H.get_bathymetry(0, 2)
    H.step_level(2, dt=dt)
    q1 = H.get_state(0, 2)
    rng = np.random.default_rng(77)
    inner = [b for b in boxes.tolist() if b[0] >= NG and b[1] >= NG and b[2] <= nf - NG and b[3] <= nf - NG]
    # the three patches with the strongest flow and three at random
    act = [np.abs(q0[[1, 2, 4, 5], b[1]:b[3], b[0]:b[2]]).max() for b in inner]
    picks = list(np.argsort(act)[-3:]) + list(rng.choice(len(inner), 3, replace=False))
    # level-wide per-field scale (momenta at least h_max sqrt(g h_max) of their layer)
    scale = np.maximum(state_scale(q0, 2), state_scale(q1, 2))
    P = O.params(M=2, dry_tol=1e-3)
    worst = np.zeros(6)
    for k in picks:
        i0, j0, i1, j1 = inner[k]
        qp = np.ascontiguousarray(q0[:, j0 - NG:j1 + NG, i0 - NG:i1 + NG])
        Bp = np.ascontiguousarray(B2[j0 - NG:j1 + NG, i0 - NG:i1 + NG])
        O.step_patch(P, qp, Bp, dx, dx, dt)
        want = qp[:, NG:-NG, NG:-NG]
        err = np.abs(q1[:, j0:j1, i0:i1] - want).max(axis=(1, 2)) / scale
        worst = np.maximum(worst, err)
        assert err.max() <= TOL, (inner[k], err)
    report("amr_level2_patches", worst)


def test_level0_step_matches_oracle_walled_step(amr_full):
    H, w = amr_full
    n0, L = w["n0"], w["L"]
    dx = L / n0
    dt = 0.4
    q0 = H.get_state(0, 0)
    B0 = H.get_bathymetry(0, 0)
    H.step_level(0, dt=dt)
    q1 = H.get_state(0, 0)
    _check_walled_step(O.params(M=2, dry_tol=1e-3), q0, B0, dx, dt, q1, np.random.default_rng(79), "level 0")


@pytest.fixture(scope="module")
def ensemble_full(mlswe_lib):
    """The ensemble workload as the benchmark builds it: 256 members, coarse U{128..512}^2,
    seeded shelves and humps, one refined level (ratio 4, seeded patches)."""
    r = 4
    members = [I.ensemble_member(k) for k in range(256)]
    cfg = mlswe_lib.Config(M=2, dry_tol=1e-3, max_levels=2, ratio=[r], regrid_interval=0, min_side=16,
                           max_side=64)
    H = mlswe_lib.Hierarchy(cfg, [(0.0, 0.0, m["L"], m["L"], m["n"], m["n"]) for m in members])
    for k, m in enumerate(members):
        nf = m["n"] * r
        xf = I.centers(0.0, m["L"], nf)
        H.set_bathymetry(k, np.ascontiguousarray(np.broadcast_to(
            I.shelf_B(xf, depth=m["depth"], shelf_x=m["shelf_x"])[None, :], (nf, nf))))
        B0 = H.get_bathymetry(k, 0)
        x0 = I.centers(0.0, m["L"], m["n"])
        X, Y = np.meshgrid(x0, x0)
        H.set_state(k, 0, I.layered_state(B0, I.hump_field(X, Y, *m["humps"]), -200.0 * np.ones_like(B0)))
        H.set_patches(k, 1, I.random_layout(5100 + k, m["n"] * r, m["n"] * r, max(4, m["n"] // 16), r))
        H.interp_fine(0, k)
    for lev in range(2):
        H.autotune(lev, iters=2)
    H.advance(1)
    yield H, members, r
    H.close()


def test_ensemble_sampled_members_match_oracle(ensemble_full):
    """One step of every member's level 0 (each with its own dt, one launch) and then of
    every member's refined level: sampled members' level 0 against the oracle's walled step,
    sampled patches of two members against the oracle's patch step."""
    H, members, r = ensemble_full
    dx0 = np.array([m["L"] / m["n"] for m in members])
    c = np.sqrt(9.81 * np.array([m["depth"] for m in members]))
    dt0 = 0.45 * dx0 / c
    P = O.params(M=2, dry_tol=1e-3)
    ns = [m["n"] for m in members]
    sample = [int(np.argmin(ns)), int(np.argmax(ns)), 97]
    q0 = {k: H.get_state(k, 0) for k in sample}
    H.step_level(0, dt=dt0)
    rng0 = np.random.default_rng(80)
    for k in sample:
        _check_walled_step(P, q0[k], H.get_bathymetry(k, 0), dx0[k], dt0[k], H.get_state(k, 0), rng0, k)
    # the refined level, from rings filled at the level-0 state just reached
    H.fill_ghosts(1, 1.0)
    rng = np.random.default_rng(78)
    before = {}
    for k in (sample[1], 5):
        nf = members[k]["n"] * r
        qa = H.get_state(k, 1)
        boxes = [b for b in H.get_patches(k, 1).tolist()
                 if b[0] >= NG and b[1] >= NG and b[2] <= nf - NG and b[3] <= nf - NG]
        picks = rng.choice(len(boxes), min(2, len(boxes)), replace=False)
        before[k] = (qa, [(boxes[i], np.ascontiguousarray(qa[:, boxes[i][1] - NG:boxes[i][3] + NG,
                                                             boxes[i][0] - NG:boxes[i][2] + NG])) for i in picks])
    H.step_level(1, dt=dt0 / r)
    for k, (qa, inputs) in before.items():
        nf = members[k]["n"] * r
        qb = H.get_state(k, 1)
        Bf = H.get_bathymetry(k, 1)
        scale = np.maximum(state_scale(qa, 2), state_scale(qb, 2))
        dxf = members[k]["L"] / nf
        worst = np.zeros(6)
        for (i0, j0, i1, j1), qp in inputs:
            Bp = np.ascontiguousarray(Bf[j0 - NG:j1 + NG, i0 - NG:i1 + NG])
            O.step_patch(P, qp, Bp, dxf, dxf, dt0[k] / r)
            want = qp[:, NG:-NG, NG:-NG]
            err = np.abs(qb[:, j0:j1, i0:i1] - want).max(axis=(1, 2)) / scale
            worst = np.maximum(worst, err)
            assert err.max() <= TOL, (k, (i0, j0, i1, j1), err)
        report(f"ensemble_member{k}_refined_patches", worst)


def test_adjoint_full_size_gradient_matches_central_fd(mlswe_lib):
    """The adjoint workload as the benchmark runs it (512^2, 200 first-order steps, 32
    gauges, checkpoints every 20, per-edge forward records kept): the gradient with respect
    to eta_1 and B along six seeded directions mixing both controls against central
    differences of the GPU forward loss."""
    import torch
    from paper_1803_01450_gb300.adjoint import FixedGridProblem, gauge_misfit
    n, steps, ckpt, n_g, L = 512, 200, 20, 32, 1e5
    B = I.adjoint_bathymetry(n, L)
    eta1 = I.adjoint_eta1(n, seed=4000, L=L)
    gauges = I.gauge_cells(n, n_g, seed=4100)
    dt = 0.5 * (L / n) / 205.0
    prob = FixedGridProblem(n, n, L, dt, steps, ckpt, gauges, np.zeros((steps, n_g)))
    dev = torch.device("cuda", 0)
    e = torch.tensor(eta1, dtype=torch.float64, device=dev, requires_grad=True)
    Bt = torch.tensor(B, dtype=torch.float64, device=dev, requires_grad=True)
    loss = gauge_misfit(e, Bt, prob)
    loss.backward()
    ge, gB = e.grad.cpu().numpy(), Bt.grad.cpu().numpy()
    assert np.abs(ge).max() > 0 and np.abs(gB).max() > 0
    rng = np.random.default_rng(10)
    x_norm = np.sqrt(np.sum(eta1 ** 2) + np.sum(B ** 2))
    for _ in range(6):
        de = rng.standard_normal(ge.shape)
        dB = rng.standard_normal(gB.shape)
        d_norm = np.sqrt(np.sum(de ** 2) + np.sum(dB ** 2))
        eps = 1e-6 * x_norm / d_norm
        Jp = prob.forward(eta1 + eps * de, B + eps * dB)
        Jm = prob.forward(eta1 - eps * de, B - eps * dB)
        fd = (Jp - Jm) / (2 * eps)
        ad = float(np.sum(ge * de) + np.sum(gB * dB))
        assert abs(fd - ad) <= 1e-6 * abs(fd), (fd, ad)
    prob.close()
