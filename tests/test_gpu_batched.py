"""Batched execution: every patch of a level of every ensemble member in one persistent
launch, whole coarse steps replayed from CUDA graphs, per-member device time steps, and the
tile autotuner. The execution form must not change any result: graph replay, direct
launches and one launch per patch give bit-identical states; the ensemble matches the
oracle member by member."""
import numpy as np
import pytest

import oracle as O
from oracle.amr import OracleAMR
from paper_1803_01450_gb300 import inputs as I
from conftest import rel_err, report, state_err, state_scale

pytestmark = pytest.mark.gpu
TOL = 1e-11


def _ensemble(pkg, members, levels=2, r=4, regrid=4):
    cfg = pkg.Config(M=2, dry_tol=1e-3, max_levels=levels, ratio=[r, r], flag_tol=2e-5, regrid_interval=regrid,
                     n_buf=2, cluster_eff=0.7, min_side=16, max_side=64)
    doms = [(0.0, 0.0, m["L"], m["L"], m["n"], m["n"]) for m in members]
    H = pkg.Hierarchy(cfg, doms)
    states = []
    for k, m in enumerate(members):
        nf = m["n"] * r ** (levels - 1)
        _, Bf = I.ensemble_state(m, nf)  # bathymetry sampled at the finest cell centres
        H.set_bathymetry(k, Bf)
        B0 = H.get_bathymetry(k, 0)
        q0 = I.layered_state(B0, _eta1(m, m["n"]), -200.0 * np.ones_like(B0))
        H.set_state(k, 0, q0)
        states.append((q0, Bf))
    return H, states


def _eta1(member, n):
    x = I.centers(0.0, member["L"], n)
    X, Y = np.meshgrid(x, x)
    return I.hump_field(X, Y, *member["humps"])


def _members(k_list, n_min=48, n_max=80):
    return [I.ensemble_member(k, n_min=n_min, n_max=n_max) for k in k_list]


def test_graph_direct_and_per_patch_are_bit_identical(mlswe_lib):
    members = _members(range(3))
    outs = []
    for mode in ("graph", "direct", "per_patch"):
        H, _ = _ensemble(mlswe_lib, members)
        if mode == "direct":
            H.set_execution(use_graphs=False)
        elif mode == "per_patch":
            H.set_execution(use_graphs=False, per_patch_launches=True)
        H.advance(9)
        outs.append([(H.get_state(k, 0), H.get_state(k, 1), H.get_patches(k, 1)) for k in range(len(members))])
        H.close()
    for k in range(len(members)):
        for mode in (1, 2):
            assert np.array_equal(outs[0][k][2], outs[mode][k][2])
            assert np.array_equal(outs[0][k][0], outs[mode][k][0])
            assert np.array_equal(outs[0][k][1], outs[mode][k][1])


@pytest.mark.parametrize("M,unsplit", [(1, 0), (3, 0), (2, 1)])
def test_packed_and_per_patch_tiles_bit_identical(mlswe_lib, M, unsplit):
    """The batched form packs runs of patch lines of several patches into one sweep tile;
    the per-patch form keeps one rectangle of one patch per tile. One layer, three layers and
    the unsplit step over two members of different sizes, regridding: identical layouts and
    bit-identical states."""
    r = 2
    sizes = [(40, 40), (56, 48)]
    rho = {1: (1000.0,), 2: (1000.0, 1025.0), 3: (1000.0, 1020.0, 1030.0)}[M]
    surfaces = [-0.4, -0.8][: M - 1]
    outs = []
    for per_patch in (False, True):
        cfg = mlswe_lib.Config(M=M, rho=rho, dry_tol=1e-6, max_levels=2, ratio=[r], flag_tol=1e-3,
                               regrid_interval=4, n_buf=2, cluster_eff=0.7, min_side=8, max_side=32,
                               unsplit=unsplit)
        H = mlswe_lib.Hierarchy(cfg, [(0.0, 0.0, 1.0, 1.0, nx, ny) for nx, ny in sizes])
        for k, (nx, ny) in enumerate(sizes):
            xf, yf = (np.arange(nx * r) + 0.5) / (nx * r), (np.arange(ny * r) + 0.5) / (ny * r)
            Xf, _ = np.meshgrid(xf, yf)
            H.set_bathymetry(k, -1.5 + 0.2 * Xf)
            B0 = H.get_bathymetry(k, 0)
            X, Y = np.meshgrid((np.arange(nx) + 0.5) / nx, (np.arange(ny) + 0.5) / ny)
            eta1 = 0.02 * np.exp(-((X - 0.3 - 0.2 * k) ** 2 + (Y - 0.5) ** 2) / 0.005)
            H.set_state(k, 0, I.stacked_state(B0, [eta1] + [s + 0.0 * X for s in surfaces]))
        if per_patch:
            H.set_execution(use_graphs=False, per_patch_launches=True)
        H.advance(8)
        outs.append([(H.get_patches(k, 1), H.get_state(k, 0), H.get_state(k, 1)) for k in range(len(sizes))])
        H.close()
    for k in range(len(sizes)):
        assert len(outs[0][k][0]) > 0
        for a, b in zip(outs[0][k], outs[1][k]):
            assert np.array_equal(a, b)


def test_graph_replay_is_deterministic(mlswe_lib):
    members = _members(range(2))
    res = []
    for _ in range(2):
        H, _ = _ensemble(mlswe_lib, members)
        H.advance(6)
        res.append(H.get_state(1, 1))
        H.close()
    assert np.array_equal(res[0], res[1])


def test_ensemble_members_match_oracle(mlswe_lib):
    """Every member of a 3-member ensemble (different grids, bathymetry, humps and time
    steps) advanced together matches its own oracle run."""
    members = _members(range(3))
    H, states = _ensemble(mlswe_lib, members)
    H.advance(8)
    t, dt = H.get_time()
    for k, m in enumerate(members):
        q0, Bf = states[k]
        P = O.params(M=2, dry_tol=1e-3)
        A = OracleAMR(P, (0, 0, m["L"], m["L"]), m["n"], m["n"], 2, [4], Bf, flag_tol=2e-5, min_side=16, max_side=64)
        A.set_state(0, q0)
        A.advance(8, regrid_interval=4)
        assert [tuple(b) for b in H.get_patches(k, 1).tolist()] == [tuple(b) for b in A.lev[1].patches]
        assert abs(t[k] - A.t) <= 1e-12 * A.t
        # momenta against at least h_max sqrt(g h_max) of their layer (state_scale)
        err = state_err(H.get_state(k, 0), A.lev[0].q, 2)
        report(f"ensemble3_member{k}_level0", err)
        assert err.max() <= TOL, (k, err)
    assert len(set(np.round(dt, 12))) == len(members)  # per-member time steps differ
    H.close()


def test_autotune_keeps_state_and_results(mlswe_lib):
    members = _members(range(2))
    H1, _ = _ensemble(mlswe_lib, members)
    H1.advance(4)
    q_before = H1.get_state(0, 1)
    chosen = H1.autotune(1, iters=2)
    assert np.array_equal(H1.get_state(0, 1), q_before)
    assert chosen[0] >= 4 and chosen[3] >= 4 and chosen[2] in (1, 2) and chosen[5] in (1, 2)
    H1.advance(4)
    H2, _ = _ensemble(mlswe_lib, members)
    H2.advance(8)
    for k in range(2):
        assert np.array_equal(H1.get_state(k, 1), H2.get_state(k, 1))
    H1.close()
    H2.close()


def test_more_members_than_one_cta(mlswe_lib):
    """1100 one-level members (the time-step kernel spans several CTAs): every member keeps
    its own time step; a sample of members matches its own oracle run."""
    n, nm = 8, 1100
    depths = 1.0 + 0.001 * np.arange(nm)
    cfg = mlswe_lib.Config(M=1, dry_tol=1e-6, max_levels=1, regrid_interval=0)
    H = mlswe_lib.Hierarchy(cfg, [(0.0, 0.0, 1.0, 1.0, n, n)] * nm)
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x)
    states = []
    for k in range(nm):
        B = -depths[k] * np.ones((n, n))
        q = np.zeros((3, n, n))
        q[0] = depths[k] + 0.01 * np.exp(-((X - 0.5) ** 2 + (Y - 0.4) ** 2) / 0.02)
        H.set_bathymetry(k, B)
        H.set_state(k, 0, q)
        states.append((B, q))
    H.advance(2)
    t, _ = H.get_time()
    assert len(set(np.round(t, 15))) == nm  # deeper members take shorter steps
    for k in (0, 517, 1024, 1099):
        B, q = states[k]
        A = OracleAMR(O.params(M=1, dry_tol=1e-6), (0, 0, 1, 1), n, n, 1, [], B)
        A.set_state(0, q)
        A.advance(2)
        assert abs(t[k] - A.t) <= 1e-12 * A.t
        assert rel_err(H.get_state(k, 0), A.lev[0].q).max() < 1e-11
    H.close()
