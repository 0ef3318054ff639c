"""The patch partition through torch.distributed as bench.py --gpus N runs it
(sharding.PatchPartition: all-gather of the packed patch values and a max-all-reduce of the
wave-speed slots inside the library's exchange hook), with two rank processes on one GPU over
the gloo backend (host-staged collectives: the processes wait for each other on the host, no
kernel waits on another). Every rank's hierarchy must equal the undivided run bit for bit, and
bench.py's partitioned AMR figure must come out on a small case.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(pkg):
    from paper_1803_01450_gb300 import inputs as I
    n = 40
    cfg = pkg.Config(M=2, dry_tol=1e-6, max_levels=3, ratio=[2, 2], flag_tol=1e-3, regrid_interval=3,
                     min_side=8, max_side=16)
    return cfg, n, I.small(n)["q"], -np.ones((4 * n, 4 * n))


def _run(pkg, stream=None, part=None):
    cfg, n, q, B = _case(pkg)
    H = pkg.Hierarchy(cfg, [(0.0, 0.0, 1.0, 1.0, n, n)], stream=stream)
    H.set_bathymetry(0, B)
    H.set_state(0, 0, q)
    if part is not None:
        part(H)
    H.advance(7)
    out = []
    for l in range(3):
        boxes = H.get_patches(0, l)
        st = H.get_state(0, l)
        if l > 0:
            m = np.zeros(st.shape[1:], bool)
            for (i0, j0, i1, j1) in boxes.tolist():
                m[j0:j1, i0:i1] = True
            st = st[:, m]
        out.append((boxes, st))
    t = H.get_time()[0]
    H.close()
    return out, t


def _worker(rank, ws, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import torch
    import torch.distributed as dist
    import paper_1803_01450_gb300 as pkg
    from paper_1803_01450_gb300 import sharding as S
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        stream = torch.cuda.Stream(device=dev)
        res, t = _run(pkg, stream.cuda_stream, lambda H: S.PatchPartition(H, rank, ws, dist, dev))
        import bench
        fig = bench.bench_amr_partitioned(pkg, torch, stream, rank, ws, steps=2, n0=128, patches=(40, 120))
        gathered = [None] * ws
        dist.all_gather_object(gathered, (rank, res, t, fig))
        if rank == 0:
            np.save(os.path.join(out_dir, "part.npy"), np.array(gathered, dtype=object), allow_pickle=True)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_patch_partition_two_processes_gloo(mlswe_lib, tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    mp.start_processes(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    gathered = np.load(tmp_path / "part.npy", allow_pickle=True)
    want, t_want = _run(mlswe_lib)
    assert len(want[2][0]) > 1
    for _, res, t, fig in gathered:
        assert np.array_equal(t, t_want)
        for (bg, qg), (bw, qw) in zip(res, want):
            assert np.array_equal(bg, bw)
            assert np.array_equal(qg, qw)
        assert fig["ranks"] == 2 and fig["lcups"] > 0
