"""The multi-GPU splits of the work (paper_1803_01450_gb300.sharding), on CPU: gloo ranks in
separate processes, the oracle as the stepping function. What the GPU path adds to a
member's step is only where its rows and members live, so every rank-split result must equal
the undivided run bit for bit:

* ensemble members partitioned across two ranks, each rank advancing its members (two-level
  AMR runs of the oracle), gathered and compared with single-process runs; the job's cell
  updates reduced with an all-reduce;
* one grid split into slabs of rows on two and three ranks, halo rows swapped by
  point-to-point sends before every step, stepped with the oracle's walled step on the local
  rows (the local array's ends act as walls, which only the halo rows see), and the owned
  rows gathered after 12 second-order steps; one time step for all slabs from the largest
  speed over every rank's owned cells (a max-all-reduce).
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1803_01450_gb300 import sharding as S  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


# ---------------------------------------------------------------------- single-process logic
def test_partition_members_covers_and_balances():
    rng = np.random.default_rng(3)
    costs = [int(c) for c in rng.integers(128, 513, 256) ** 2]
    for ws in (1, 2, 3, 8):
        parts = S.partition_members(costs, ws)
        flat = sorted(k for p in parts for k in p)
        assert flat == list(range(256))
        loads = [sum(costs[k] for k in p) for p in parts]
        assert max(loads) - min(loads) <= max(costs)  # greedy largest-first bound
        assert parts == S.partition_members(costs, ws)  # deterministic
        assert all(p == sorted(p) for p in parts)


def test_slabs_cover_rows_with_halos():
    for ny, ws in ((37, 2), (64, 3), (2048, 8), (9, 4)):
        slabs = [S.slab_of(ny, ws, r) for r in range(ws)]
        assert slabs[0].j0 == 0 and slabs[-1].j1 == ny
        for a, b in zip(slabs, slabs[1:]):
            assert a.j1 == b.j0 and a.hi == a.j1 + S.HALO and b.lo == b.j0 - S.HALO
        assert slabs[0].lo == 0 and slabs[-1].hi == ny
        assert max(s.j1 - s.j0 for s in slabs) - min(s.j1 - s.j0 for s in slabs) <= 1
    with pytest.raises(ValueError):
        S.slab_of(5, 4, 0)


# ---------------------------------------------------------------------- gloo ranks
def _members():
    from paper_1803_01450_gb300 import inputs as I
    out = []
    for k in range(5):
        n = 24 + 8 * k
        w = I.small(n)
        out.append((n, w["q"]))
    return out


def _run_member(n, q, steps=6):
    import oracle as O
    from oracle.amr import OracleAMR
    P = O.params(M=2, dry_tol=1e-6)
    A = OracleAMR(P, (0, 0, 1, 1), n, n, 2, [2], -np.ones((2 * n, 2 * n)), min_side=8, max_side=32)
    A.set_state(0, q)
    A.advance(steps, regrid_interval=3)
    cells = sum(s * sum((b[2] - b[0]) * (b[3] - b[1]) for b in V.patches)
                for s, V in zip(A.level_steps, A.lev))
    return A.lev[0].q, A.lev[1].q, A.t, cells


def _slab_case():
    from paper_1803_01450_gb300 import inputs as I
    ny, nx = 41, 29
    q, B = I.gaussian_random_state(71, 2, nx, ny)
    return q, B, 1.0 / nx, 1.2 / ny


def _slab_run(rank, ws, dist, steps=12):
    """Each rank steps its slab with halo swaps; returns its owned rows and the time."""
    import torch
    import oracle as O
    q, B, dx, dy = _slab_case()
    ny = q.shape[1]
    P = O.params(M=2, dry_tol=1e-6, order=2, limiter=2)
    sl = S.slab_of(ny, ws, rank)
    loc = q[:, sl.lo:sl.hi].copy()
    Bl = np.ascontiguousarray(B[:, :][sl.lo:sl.hi])
    F = q.shape[0]

    def get_rows(r0, n):
        return torch.from_numpy(np.ascontiguousarray(loc[:, r0:r0 + n]))

    def set_rows(r0, n, t):
        loc[:, r0:r0 + n] = t.numpy().reshape(F, n, -1)

    t = 0.0
    for k in range(steps):
        S.halo_exchange(sl, rank, ws, get_rows, set_rows, dist)
        # one time step for all slabs: the largest speed over every rank's owned cells
        dt = 0.8 * min(dx, dy) / S.max_all(_speed(loc[:, sl.own]), dist)
        new, _, _ = O.step_walled(P, loc, Bl, dx, dy, dt)
        loc[:] = new
        t += dt
    return loc[:, sl.own].copy(), t


def _speed(q, g=9.81):
    """Largest max_m(|u_m|, |v_m|) + sqrt(g sum_m h_m) over the cells of q (two layers)."""
    h = q[0] + q[3]
    u = np.maximum.reduce([np.abs(q[3 * m + k]) / q[3 * m] for m in range(2) for k in (1, 2)])
    return float((u + np.sqrt(g * h)).max())


def _single_slab_run(steps=12):
    import oracle as O
    q, B, dx, dy = _slab_case()
    P = O.params(M=2, dry_tol=1e-6, order=2, limiter=2)
    t = 0.0
    for k in range(steps):
        dt = 0.8 * min(dx, dy) / _speed(q)
        q, _, _ = O.step_walled(P, q, B, dx, dy, dt)
        t += dt
    return q, t


def _worker(rank, ws, port, out_dir, what):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        if what == "members":
            members = _members()
            parts = S.partition_members([n * n for n, _ in members], ws)
            mine = {k: _run_member(*members[k]) for k in parts[rank]}
            total = S.sum_all(sum(r[3] for r in mine.values()), dist)
            gathered = [None] * ws
            dist.all_gather_object(gathered, {k: v[:3] for k, v in mine.items()})
            if rank == 0:
                allres = {}
                for g in gathered:
                    allres.update(g)
                np.save(os.path.join(out_dir, "members.npy"), np.array([allres, total, parts], dtype=object),
                        allow_pickle=True)
        else:
            if what == "slabs_halo1":
                S.HALO = 1  # planted: one halo row where the stencil reaches two
            own, t = _slab_run(rank, ws, dist)
            gathered = [None] * ws
            dist.all_gather_object(gathered, (rank, own, t))
            if rank == 0:
                np.save(os.path.join(out_dir, "slabs.npy"), np.array(gathered, dtype=object), allow_pickle=True)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _spawn(ws, tmp_path, what):
    mp = pytest.importorskip("torch.multiprocessing")
    mp.start_processes(_worker, args=(ws, _free_port(), str(tmp_path), what), nprocs=ws, join=True,
                       start_method="spawn")


def test_members_partitioned_over_two_ranks_equal_single_process(tmp_path):
    _spawn(2, tmp_path, "members")
    allres, total, parts = np.load(tmp_path / "members.npy", allow_pickle=True)
    members = _members()
    assert sorted(allres) == list(range(len(members))) and all(len(p) > 0 for p in parts)
    want_total = 0
    for k, (n, q) in enumerate(members):
        q0, q1, t, cells = _run_member(n, q)
        want_total += cells
        assert np.array_equal(allres[k][0], q0) and np.array_equal(allres[k][1], q1) and allres[k][2] == t
    assert total == want_total


@pytest.mark.parametrize("ws", [2, 3])
def test_slabs_with_halo_swaps_equal_undivided_grid(tmp_path, ws):
    _spawn(ws, tmp_path, "slabs")
    gathered = sorted(np.load(tmp_path / "slabs.npy", allow_pickle=True), key=lambda g: g[0])
    want, t_want = _single_slab_run()
    got = np.concatenate([g[1] for g in gathered], axis=1)
    assert all(g[2] == t_want for g in gathered)
    assert np.array_equal(got, want)


def test_planted_one_row_halo_fails(tmp_path):
    """With one halo row the second-order stencil of the rows next to a slab edge reads a cell
    the swap never refreshed: the slabs no longer equal the undivided grid."""
    _spawn(2, tmp_path, "slabs_halo1")
    gathered = sorted(np.load(tmp_path / "slabs.npy", allow_pickle=True), key=lambda g: g[0])
    want, _ = _single_slab_run()
    got = np.concatenate([g[1] for g in gathered], axis=1)
    assert got.shape == want.shape and not np.array_equal(got, want)
