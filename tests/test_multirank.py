"""Host logic of the multi-rank benchmark path, on CPU with the gloo backend and two ranks:
each rank advances its own replica (independent problems, no data-path collective), the
timed region is the slowest rank's, the job value counts the units of every rank, and the
oracle arm runs on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import torch
    import torch.distributed as dist
    import bench
    from paper_1803_01450_gb300 import inputs as I

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    # replicas: rank-seeded inputs differ between ranks
    q = I.scale(32, seed=bench.replica_seed(rank))["q"]
    sums = [torch.zeros(1, dtype=torch.float64) for _ in range(ws)]
    dist.all_gather(sums, torch.tensor([float(np.abs(q).sum())], dtype=torch.float64))
    # the slowest rank's time, seen by every rank
    ms_local = 10.0 * (rank + 1)
    tmax = bench.max_over_ranks(ms_local, ws)
    value = bench.job_value(1000.0, 5, ws, tmax)
    # the oracle arm: ranks other than 0 do no work and print nothing
    printed = ""
    if rank != 0:
        buf = io.StringIO()
        with redirect_stdout(buf):
            bench.run_reference(type("A", (), {"steps": 1, "warmup": 0})())
        printed = buf.getvalue()
    dist.barrier()
    dist.destroy_process_group()
    np.save(os.path.join(out_dir, f"r{rank}.npy"),
            np.array([tmax, value, sums[0].item(), sums[1].item(), len(printed)], dtype=np.float64))


def test_two_rank_replicas_and_timing(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    ws, port = 2, _free_port()
    mp.start_processes(_worker, args=(ws, port, str(tmp_path)), nprocs=ws, join=True, start_method="spawn")
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    assert r0[0] == r1[0] == 20.0                     # max over ranks
    assert r0[1] == r1[1] == 1000.0 * 5 * 2 / 0.020   # every rank's units over the slowest time
    assert r0[2] == r1[2] and r0[3] == r1[3]          # same gathered checksums on both ranks
    assert r0[2] != r0[3]                             # different replicas per rank
    assert r1[4] == 0                                 # rank 1 printed nothing in the oracle arm
