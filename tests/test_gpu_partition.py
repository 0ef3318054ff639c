"""Patches of the refined levels split over ranks (mlswe_set_partition), emulated on one GPU in
one process: each rank is a hierarchy advanced by its own host thread on its own stream, and
the exchange hook moves the packed patch values and the wave-speed slots between the
hierarchies through device copies, with host barriers between the phases (no kernel waits on
another). After the runs every rank's hierarchy must equal the undivided one bit for bit:
every level's patch cells, the layouts the regrids chose, the times. The finest level
moves in pieces (halo cells between substeps, halo cells and reflux accumulators after the
last, the parent cells each rank coarsened, the whole level only before regrids and at the
end of advance); the bit-for-bit equality checks that nothing else is read meanwhile.

* three levels (ratios 2, 2) with regrids, two and three ranks;
* two members with ratios 4, 4 and the dynamic time ratio, two ranks;
* three layers, ratio 4, three ranks;
* four ranks for two patches (ranks with nothing to sweep or send);
* a coarse step forced above cfl_max, rejected and retaken alike on every rank;
* the library's owners equal the restated rule (sharding.partition_patches);
* refusals: a bad rank, the per-patch launch form while partitioned.
"""
import threading

import numpy as np
import pytest

from paper_1803_01450_gb300 import inputs as I
from paper_1803_01450_gb300 import sharding as S

pytestmark = pytest.mark.gpu


class _Group:
    def __init__(self, ws):
        self.ws = ws
        self.barrier = threading.Barrier(ws, timeout=300)
        self.bufs = [None] * ws
        self.speeds = [None] * ws
        self.calls = [0] * ws
        self.modes = [0, 0, 0, 0]  # rank 0's exchanges by kind (full, halo, last, averaged)


def _hook(H, r, grp, dev):
    import torch

    def hook(level, kind):
        stream = torch.cuda.ExternalStream(H.stream, device=dev)
        sizes = H.partition_sizes(level, kind)
        grp.modes[kind] += 1 if r == 0 else 0
        with torch.cuda.stream(stream):
            buf = torch.empty(max(max(sizes), 1), dtype=torch.float64, device=dev)
            if sizes[r] > 0:
                H.partition_pack(level, buf.data_ptr(), kind)
            ptr, n = H.wave_speed_slots()
            sp = torch.as_tensor(S._DeviceArray(ptr, n), device=dev)
            snap = sp.clone()
        stream.synchronize()
        grp.bufs[r], grp.speeds[r] = buf, snap
        grp.calls[r] += 1
        grp.barrier.wait()
        with torch.cuda.stream(stream):
            for q in range(grp.ws):
                if q != r and sizes[q] > 0:
                    H.partition_unpack(level, q, grp.bufs[q].data_ptr(), kind)
            sp.copy_(torch.stack(grp.speeds).amax(dim=0))
        stream.synchronize()
        grp.barrier.wait()

    return hook


def _make(pkg, cfg, members, stream=None):
    H = pkg.Hierarchy(cfg, [(0.0, 0.0, 1.0, 1.0, n, n) for n, _, _ in members], stream=stream)
    for k, (n, q, B) in enumerate(members):
        H.set_bathymetry(k, B)
        H.set_state(k, 0, q)
    return H


def _snapshot(H, n_members, L):
    out = []
    for k in range(n_members):
        levels = []
        for l in range(L):
            boxes = H.get_patches(k, l)
            q = H.get_state(k, l)
            if l == 0:
                levels.append((boxes, q))
            else:
                m = np.zeros(q.shape[1:], bool)
                for (i0, j0, i1, j1) in boxes.tolist():
                    m[j0:j1, i0:i1] = True
                levels.append((boxes, q[:, m]))
        out.append(levels)
    return out, H.get_time()[0]


def _run_partitioned(pkg, cfg, members, ws, steps, L):
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    grp = _Group(ws)
    streams = [torch.cuda.Stream(device=dev) for _ in range(ws)]
    hs = [_make(pkg, cfg, members, stream=streams[r].cuda_stream) for r in range(ws)]
    for r, H in enumerate(hs):
        H.set_partition(r, ws, _hook(H, r, grp, dev))
    errors = [None] * ws

    def run(r):
        try:
            hs[r].advance(steps)
        except BaseException as e:  # reported below
            errors[r] = e
            grp.barrier.abort()

    threads = [threading.Thread(target=run, args=(r,)) for r in range(ws)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for e in errors:
        if e is not None:
            raise e
    owners = [[H.partition_owners(k, l) for l in range(1, L) for k in range(len(members))] for H in hs]
    snaps = [_snapshot(H, len(members), L) for H in hs]
    layouts = [[H.get_patches(k, l) for k in range(len(members))] for l in range(1, L) for H in hs[:1]]
    for H in hs:
        H.close()
    return snaps, owners, layouts, grp.calls


def _assert_equal(snap, want):
    (levels_got, t_got), (levels_want, t_want) = snap, want
    assert np.array_equal(t_got, t_want)
    for mg, mw in zip(levels_got, levels_want):
        for (bg, qg), (bw, qw) in zip(mg, mw):
            assert np.array_equal(bg, bw)
            assert np.array_equal(qg, qw)


def _three_level_case():
    n = 40
    w = I.small(n)
    return [(n, w["q"], -np.ones((4 * n, 4 * n)))]


@pytest.mark.parametrize("ws", [2, 3])
def test_three_levels_partitioned_equal_undivided(mlswe_lib, ws):
    pkg = mlswe_lib
    cfg = pkg.Config(M=2, dry_tol=1e-6, max_levels=3, ratio=[2, 2], flag_tol=1e-3, regrid_interval=3,
                     min_side=8, max_side=16)
    members = _three_level_case()
    H = _make(pkg, cfg, members)
    H.regrid(0)
    H.advance(7)
    want = _snapshot(H, 1, 3)
    H.close()
    assert len(want[0][0][2][0]) > 1  # several level-2 patches to split

    # the partitioned runs start from the same regridded layout
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    grp = _Group(ws)
    streams = [torch.cuda.Stream(device=dev) for _ in range(ws)]
    hs = [_make(pkg, cfg, members, stream=streams[r].cuda_stream) for r in range(ws)]
    for r, Hr in enumerate(hs):
        Hr.regrid(0)
        Hr.set_partition(r, ws, _hook(Hr, r, grp, dev))
    errors = [None] * ws

    def run(r):
        try:
            hs[r].advance(7)
        except BaseException as e:
            errors[r] = e
            grp.barrier.abort()

    threads = [threading.Thread(target=run, args=(r,)) for r in range(ws)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for e in errors:
        if e is not None:
            raise e
    for l in (1, 2):
        own = hs[0].partition_owners(0, l)
        assert own.tolist() == S.partition_patches([hs[0].get_patches(0, l).tolist()], ws)[0]
        assert set(own.tolist()) == set(range(ws))  # every rank sweeps something
    snaps = [_snapshot(Hr, 1, 3) for Hr in hs]
    for Hr in hs:
        Hr.close()
    assert min(grp.calls) > 0 and len(set(grp.calls)) == 1
    assert min(grp.modes) > 0  # every kind of exchange ran
    for snap in snaps:
        _assert_equal(snap, want)


def test_two_members_dynamic_ratio_partitioned_equal_undivided(mlswe_lib):
    pkg = mlswe_lib
    cfg = pkg.Config(M=2, dry_tol=1e-6, max_levels=3, ratio=[4, 4], flag_tol=1e-3, regrid_interval=2,
                     min_side=8, max_side=24, dynamic_rt=1)
    members = []
    for k, n in enumerate((24, 32)):
        w = I.small(n)
        members.append((n, w["q"], -np.ones((16 * n, 16 * n))))
    H = _make(pkg, cfg, members)
    H.advance(5)
    want = _snapshot(H, 2, 3)
    H.close()
    snaps, owners, _, calls = _run_partitioned(pkg, cfg, members, 2, 5, 3)
    assert min(calls) > 0
    for snap in snaps:
        _assert_equal(snap, want)
    assert all(np.array_equal(a, b) for a, b in zip(owners[0], owners[1]))


def test_three_layers_partitioned_equal_undivided(mlswe_lib):
    """Three layers (the general M-layer branch and the pack layout of 9 fields), two levels
    with ratio 4 and regrids, three ranks."""
    pkg = mlswe_lib
    n = 32
    rho = (1000.0, 1020.0, 1030.0)
    cfg = pkg.Config(M=3, rho=rho, dry_tol=1e-6, max_levels=2, ratio=[4], flag_tol=1e-3, regrid_interval=2,
                     min_side=8, max_side=32)
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x)
    eta = 0.02 * np.exp(-((X - 0.45) ** 2 + (Y - 0.5) ** 2) / 0.006)
    q = np.zeros((9, n, n))
    q[6] = 0.4       # bottom layer: -1 .. -0.6
    q[3] = 0.3       # middle layer: -0.6 .. -0.3
    q[0] = 0.3 + eta  # top layer: -0.3 .. eta
    members = [(n, q, -np.ones((4 * n, 4 * n)))]
    H = _make(pkg, cfg, members)
    H.advance(5)
    want = _snapshot(H, 1, 2)
    H.close()
    assert len(want[0][0][1][0]) > 2
    snaps, _, _, calls = _run_partitioned(pkg, cfg, members, 3, 5, 2)
    assert min(calls) > 0
    for snap in snaps:
        _assert_equal(snap, want)


def test_more_ranks_than_patches(mlswe_lib):
    """Four ranks, two level-1 patches set by hand (no regrid): two ranks own no patch (empty
    sweeps and packed buffers), the run still equals the undivided one."""
    import torch
    pkg = mlswe_lib
    n = 32
    w = I.small(n)
    cfg = pkg.Config(M=2, dry_tol=1e-6, max_levels=2, ratio=[2], regrid_interval=0, min_side=8, max_side=32)
    boxes = np.array([[8, 8, 32, 40], [32, 8, 56, 24]], dtype=np.int32)

    def make(stream=None):
        H = pkg.Hierarchy(cfg, [(0.0, 0.0, 1.0, 1.0, n, n)], stream=stream)
        H.set_bathymetry(0, -np.ones((2 * n, 2 * n)))
        H.set_state(0, 0, w["q"])
        H.set_patches(0, 1, boxes)
        H.interp_fine(0, 0)
        return H

    H = make()
    H.advance(4)
    want = _snapshot(H, 1, 2)
    H.close()
    ws = 4
    dev = torch.device("cuda", torch.cuda.current_device())
    grp = _Group(ws)
    streams = [torch.cuda.Stream(device=dev) for _ in range(ws)]
    hs = [make(streams[r].cuda_stream) for r in range(ws)]
    for r, Hr in enumerate(hs):
        Hr.set_partition(r, ws, _hook(Hr, r, grp, dev))
    owners = hs[0].partition_owners(0, 1).tolist()
    assert len(set(owners)) == 2 and owners == S.partition_patches([boxes.tolist()], ws)[0]
    assert sum(1 for x in hs[0].partition_sizes(1) if x == 0) == 2
    errors = [None] * ws

    def run(r):
        try:
            hs[r].advance(4)
        except BaseException as e:
            errors[r] = e
            grp.barrier.abort()

    threads = [threading.Thread(target=run, args=(r,)) for r in range(ws)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for e in errors:
        if e is not None:
            raise e
    snaps = [_snapshot(Hr, 1, 2) for Hr in hs]
    for Hr in hs:
        Hr.close()
    for snap in snaps:
        _assert_equal(snap, want)


def _scale_speeds(H, scale):
    """The wave speeds the next time step comes from, times scale (through the clock record):
    a scale below one makes the next attempt exceed cfl_max."""
    c = H.get_clock()
    n, L = H.n_members, H.cfg.max_levels
    c[n:n + 2 * n * L] *= scale
    H.set_clock(c)


def test_courant_retakes_partitioned_equal_undivided(mlswe_lib):
    """A coarse step forced above cfl_max (speeds scaled to 40 % before it) is rejected and
    retaken on every rank alike: the ranks' Courant decisions come from the max-reduced speeds,
    the restores and retakes run on their own hierarchies, and they end equal to the undivided
    run, with the same rejection count."""
    import torch
    pkg = mlswe_lib
    cfg = pkg.Config(M=2, dry_tol=1e-6, max_levels=3, ratio=[2, 2], flag_tol=1e-3, regrid_interval=3,
                     min_side=8, max_side=16)
    members = _three_level_case()
    H = _make(pkg, cfg, members)
    H.advance(2)
    _scale_speeds(H, 0.4)
    H.advance(3)
    want = _snapshot(H, 1, 3)
    rejected = H.get_stats()["cfl_exceeded"]
    H.close()
    assert rejected > 0
    ws = 2
    dev = torch.device("cuda", torch.cuda.current_device())
    grp = _Group(ws)
    streams = [torch.cuda.Stream(device=dev) for _ in range(ws)]
    hs = [_make(pkg, cfg, members, stream=streams[r].cuda_stream) for r in range(ws)]
    for r, Hr in enumerate(hs):
        Hr.set_partition(r, ws, _hook(Hr, r, grp, dev))
    errors = [None] * ws

    def run(r, k):
        try:
            hs[r].advance(k)
        except BaseException as e:
            errors[r] = e
            grp.barrier.abort()

    for k, scale in ((2, 0.4), (3, None)):
        threads = [threading.Thread(target=run, args=(r, k)) for r in range(ws)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        for e in errors:
            if e is not None:
                raise e
        if scale is not None:
            for Hr in hs:
                _scale_speeds(Hr, scale)
    snaps = [_snapshot(Hr, 1, 3) for Hr in hs]
    counts = [Hr.get_stats()["cfl_exceeded"] for Hr in hs]
    for Hr in hs:
        Hr.close()
    assert counts == [rejected] * ws
    for snap in snaps:
        _assert_equal(snap, want)


def test_partition_refusals(mlswe_lib):
    pkg = mlswe_lib
    cfg = pkg.Config(M=2, dry_tol=1e-6, max_levels=2, ratio=[2])
    H = pkg.Hierarchy(cfg, [(0.0, 0.0, 1.0, 1.0, 16, 16)])
    for rank, ws in ((2, 2), (-1, 2), (0, 0)):
        with pytest.raises(pkg.MLSWEError) as e:
            H.set_partition(rank, ws)
        assert e.value.status == 1
    H.set_partition(1, 2)
    with pytest.raises(pkg.MLSWEError):
        H.set_execution(use_graphs=True, per_patch_launches=True)
    with pytest.raises(pkg.MLSWEError):
        H.partition_sizes(0)  # level 0 is not partitioned
    H.set_partition(0, 1)
    H.set_execution(use_graphs=True, per_patch_launches=True)
    H.close()
