"""The multi-GPU splits on one GPU, in one process (host-ordered, no kernel waits on another):
the pieces a rank would hold are separate hierarchies on one stream, and their halo rows move
through the library's device row copies (mlswe_get_rows_device / mlswe_set_rows_device) as
a rank's would move through NCCL. Results must equal the undivided runs bit for bit.

* one 2-layer grid split into two and three slabs of rows (two halo rows per shared edge),
  12 second-order steps;
* an ensemble of six members split over two hierarchies by sharding.partition_members,
  against one hierarchy of all six (subcycled AMR with regrids).
"""
import numpy as np
import pytest

from paper_1803_01450_gb300 import inputs as I
from paper_1803_01450_gb300 import sharding as S

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("ws", [2, 3])
def test_slabs_with_device_halo_copies_equal_undivided_grid(mlswe_lib, ws):
    import torch
    pkg = mlswe_lib
    ny, nx = 67, 45
    q, B = I.gaussian_random_state(91, 2, nx, ny)
    dx, dy = 1.0 / nx, 1.1 / ny
    dts = [0.2 * min(dx, dy) / 4.0 * (1.0 + 0.05 * k) for k in range(12)]
    cfg = pkg.Config(M=2, dry_tol=1e-6, order=2, limiter=2, max_levels=1)
    stream = torch.cuda.Stream()
    H = pkg.Hierarchy(cfg, [(0.0, 0.0, nx * dx, ny * dy, nx, ny)], stream=stream.cuda_stream)
    H.set_bathymetry(0, B)
    H.set_state(0, 0, q)
    for dt in dts:
        H.step_level(0, dt=dt)
    want = H.get_state(0, 0)
    H.close()

    slabs = [S.slab_of(ny, ws, r) for r in range(ws)]
    parts = []
    for sl in slabs:
        h = pkg.Hierarchy(cfg, [(0.0, 0.0, nx * dx, sl.rows * dy, nx, sl.rows)], stream=stream.cuda_stream)
        h.set_bathymetry(0, np.ascontiguousarray(B[sl.lo:sl.hi]))
        h.set_state(0, 0, np.ascontiguousarray(q[:, sl.lo:sl.hi]))
        parts.append(h)
    dev = torch.device("cuda", torch.cuda.current_device())
    buf = [torch.empty((6, S.HALO, nx), dtype=torch.float64, device=dev) for _ in range(2 * ws)]
    for dt in dts:
        # every rank's outgoing rows first, then the incoming ones (all on one stream)
        for r, (h, sl) in enumerate(zip(parts, slabs)):
            if r > 0:
                h.get_rows_device(0, 0, sl.j0 - sl.lo, S.HALO, buf[2 * r].data_ptr())
            if r < ws - 1:
                h.get_rows_device(0, 0, sl.j1 - sl.lo - S.HALO, S.HALO, buf[2 * r + 1].data_ptr())
        for r, (h, sl) in enumerate(zip(parts, slabs)):
            if r > 0:
                h.set_rows_device(0, 0, 0, S.HALO, buf[2 * (r - 1) + 1].data_ptr())
            if r < ws - 1:
                h.set_rows_device(0, 0, sl.j1 - sl.lo, S.HALO, buf[2 * (r + 1)].data_ptr())
        for h in parts:
            h.step_level(0, dt=dt)
    got = np.concatenate([h.get_state(0, 0)[:, sl.own] for h, sl in zip(parts, slabs)], axis=1)
    for h in parts:
        h.close()
    assert np.array_equal(got, want)


def test_rows_device_rejects_bad_arguments(mlswe_lib):
    pkg = mlswe_lib
    cfg = pkg.Config(M=2, dry_tol=1e-6, max_levels=1)
    H = pkg.Hierarchy(cfg, [(0.0, 0.0, 1.0, 1.0, 16, 16)])
    host = np.zeros((6, 2, 16))
    for fn in (lambda: H.get_rows_device(0, 0, 0, 2, host.ctypes.data),
               lambda: H.set_rows_device(0, 0, 15, 2, host.ctypes.data)):
        with pytest.raises(pkg.MLSWEError) as e:
            fn()
        assert e.value.status == 1
    H.close()


def test_members_partitioned_over_two_hierarchies_equal_one(mlswe_lib):
    pkg = mlswe_lib
    members = [I.small(24 + 8 * k) for k in range(6)]
    ns = [24 + 8 * k for k in range(6)]
    cfg = pkg.Config(M=2, dry_tol=1e-6, max_levels=2, ratio=[2], flag_tol=1e-3, regrid_interval=3, n_buf=2,
                     cluster_eff=0.7, min_side=8, max_side=32)

    def run(idx):
        H = pkg.Hierarchy(cfg, [(0.0, 0.0, 1.0, 1.0, ns[k], ns[k]) for k in idx])
        for j, k in enumerate(idx):
            H.set_bathymetry(j, -np.ones((2 * ns[k], 2 * ns[k])))
            H.set_state(j, 0, members[k]["q"])
        H.advance(6)
        t, _ = H.get_time()
        out = {k: (H.get_state(j, 0), H.get_state(j, 1), H.get_patches(j, 1), t[j]) for j, k in enumerate(idx)}
        cells = sum(H.get_stats()["cell_updates"])
        H.close()
        return out, cells

    whole, cells_whole = run(list(range(6)))
    parts = S.partition_members([n * n for n in ns], 2)
    split = [run(p) for p in parts]
    assert cells_whole == sum(c for _, c in split)
    for res, _ in split:
        for k, (q0, q1, boxes, t) in res.items():
            w0, w1, wb, wt = whole[k]
            assert np.array_equal(boxes, wb) and t == wt
            assert np.array_equal(q0, w0)
            m = np.zeros(q1.shape[1:], bool)
            for (i0, j0, i1, j1) in boxes.tolist():
                m[j0:j1, i0:i1] = True
            assert np.array_equal(q1[:, m], w1[:, m])
