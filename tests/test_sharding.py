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


def _boxes(seed=5, n=40, nx=96, ny=80):
    """Disjoint boxes of sides 4..16 on an nx x ny grid (seeded, placed by rejection), some of
    them touching: a refined level's patches."""
    rng = np.random.default_rng(seed)
    occ = np.zeros((ny, nx), bool)
    out = []
    while len(out) < n:
        w, h = (int(v) for v in rng.integers(4, 17, 2))
        i0, j0 = int(rng.integers(0, nx - w + 1)), int(rng.integers(0, ny - h + 1))
        if not occ[j0:j0 + h, i0:i0 + w].any():
            occ[j0:j0 + h, i0:i0 + w] = True
            out.append((i0, j0, i0 + w, j0 + h))
    return out


def test_morton_key_interleaves_bits():
    assert S.morton(0, 0) == 0 and S.morton(1, 0) == 1 and S.morton(0, 1) == 2 and S.morton(3, 5) == 39
    assert S.morton(2 ** 20, 0) == 2 ** 40 and S.morton(0, 2 ** 20) == 2 ** 41
    # Z order: the four quadrants of a 2^k square come one after another
    keys = {(i, j): S.morton(i, j) for i in range(8) for j in range(8)}
    quad = lambda i, j: (j // 4) * 2 + i // 4  # noqa: E731
    order = sorted(keys, key=keys.get)
    assert [quad(i, j) for i, j in order] == sorted(quad(i, j) for i, j in order)


def test_partition_patches_covers_balances_and_follows_the_curve():
    layouts = [_boxes(5), _boxes(6, n=25), []]
    cells = [[(b[2] - b[0]) * (b[3] - b[1]) for b in L] for L in layouts]
    biggest = max(c for cs in cells for c in cs)
    total = sum(sum(cs) for cs in cells)
    for ws in (1, 2, 3, 7):
        owners = S.partition_patches(layouts, ws)
        assert owners == S.partition_patches(layouts, ws)
        assert [len(o) for o in owners] == [len(L) for L in layouts]
        load = [0] * ws
        seq = []
        for m, L in enumerate(layouts):
            for p, b in sorted(enumerate(L), key=lambda e: (S.morton((e[1][0] + e[1][2]) // 2,
                                                                     (e[1][1] + e[1][3]) // 2), e[0])):
                load[owners[m][p]] += cells[m][p]
                seq.append(owners[m][p])
        assert seq == sorted(seq)  # contiguous runs of the curve, in rank order
        assert all(abs(x - total / ws) <= biggest for x in load)
    assert S.partition_patches([[]], 4) == [[]]


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


def _patch_case():
    rng = np.random.default_rng(17)
    ny, nx = 80, 96
    return rng.standard_normal((ny, nx)), _boxes(7, n=30, nx=nx, ny=ny)


def _patch_step(Q, boxes):
    """New values of the cells of the given boxes from Q (all from the old Q): a 5-point
    average reading the ring cells around each box (edges clamped), and the largest |value|."""
    P = np.pad(Q, 1, mode="edge")
    new, smax = [], 0.0
    for (i0, j0, i1, j1) in boxes:
        c = P[j0 + 1:j1 + 1, i0 + 1:i1 + 1]
        v = 0.5 * c + 0.125 * (P[j0:j1, i0 + 1:i1 + 1] + P[j0 + 2:j1 + 2, i0 + 1:i1 + 1]
                               + P[j0 + 1:j1 + 1, i0:i1] + P[j0 + 1:j1 + 1, i0 + 2:i1 + 2])
        new.append(v)
        smax = max(smax, float(np.abs(v).max()))
    return new, smax


def _patch_run_single(steps=6):
    Q, boxes = _patch_case()
    speeds = []
    for _ in range(steps):
        new, smax = _patch_step(Q, boxes)
        for (i0, j0, i1, j1), v in zip(boxes, new):
            Q[j0:j1, i0:i1] = v
        speeds.append(smax)
    return Q, speeds


def _patch_run_rank(rank, ws, dist, steps=6, exchange=True):
    """Each rank steps only its own boxes, then exchange_level gives it the others' cells and
    the largest |value| over the ranks."""
    import torch
    Q, boxes = _patch_case()
    owner = S.partition_patches([boxes], ws)[0]
    mine = [k for k in range(len(boxes)) if owner[k] == rank]
    cells = lambda k: (boxes[k][2] - boxes[k][0]) * (boxes[k][3] - boxes[k][1])  # noqa: E731
    sizes = [sum(cells(k) for k in range(len(boxes)) if owner[k] == r) for r in range(ws)]
    speeds = []
    for _ in range(steps):
        new, smax = _patch_step(Q, [boxes[k] for k in mine])
        for k, v in zip(mine, new):
            i0, j0, i1, j1 = boxes[k]
            Q[j0:j1, i0:i1] = v
        sp = torch.tensor([smax], dtype=torch.float64)

        def pack(buf):
            flat = np.concatenate([Q[boxes[k][1]:boxes[k][3], boxes[k][0]:boxes[k][2]].ravel() for k in mine]
                                  or [np.zeros(0)])
            buf[:flat.size] = torch.from_numpy(flat)

        def unpack(q, buf):
            o = 0
            b = buf.numpy()
            for k in range(len(boxes)):
                if owner[k] != q:
                    continue
                i0, j0, i1, j1 = boxes[k]
                Q[j0:j1, i0:i1] = b[o:o + cells(k)].reshape(j1 - j0, i1 - i0)
                o += cells(k)

        if exchange:
            S.exchange_level(rank, ws, sizes, pack, unpack, sp, dist,
                             lambda n: torch.zeros(n, dtype=torch.float64))
        else:
            dist.all_reduce(sp, op=dist.ReduceOp.MAX)
        speeds.append(float(sp[0]))
    return Q, speeds


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
        elif what in ("patches", "patches_no_exchange"):
            Q, speeds = _patch_run_rank(rank, ws, dist, exchange=(what == "patches"))
            gathered = [None] * ws
            dist.all_gather_object(gathered, (rank, Q, speeds))
            if rank == 0:
                np.save(os.path.join(out_dir, "patches.npy"), np.array(gathered, dtype=object), allow_pickle=True)
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


@pytest.mark.parametrize("ws", [2, 3])
def test_patches_partitioned_with_exchange_equal_undivided(tmp_path, ws):
    """Every rank steps its own boxes of a refined level (owners by partition_patches), then
    all-gathers the packed cells and takes the largest speed (exchange_level): every rank's
    whole array equals the undivided run's, step after step, and so do the speeds."""
    _spawn(ws, tmp_path, "patches")
    gathered = np.load(tmp_path / "patches.npy", allow_pickle=True)
    want, speeds = _patch_run_single()
    for _, Q, sp in gathered:
        assert np.array_equal(Q, want)
        assert sp == speeds


def test_planted_missing_exchange_fails(tmp_path):
    """Without the all-gather each rank's ring cells from the other ranks' boxes go stale."""
    _spawn(2, tmp_path, "patches_no_exchange")
    gathered = np.load(tmp_path / "patches.npy", allow_pickle=True)
    want, _ = _patch_run_single()
    assert not all(np.array_equal(Q, want) for _, Q, _ in gathered)
