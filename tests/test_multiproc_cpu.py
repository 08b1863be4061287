"""The multi-process side of bench.py on CPU (gloo, world size 2): every rank
solves its own batch (different seeds, weak scaling) and the job time is the
maximum over ranks.  The GPU path runs the same functions over NCCL."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        t = bench.max_over_ranks(10.0 + rank, torch.device("cpu"), dist)
        pts = [p for p, _ in bench.rank_workloads(rank, 2)]
        digest = float(sum(np.abs(p).sum() for p in pts))
        out[rank] = (t, digest)
    finally:
        dist.destroy_process_group()


def test_bench_ranks_max_time_and_distinct_batches():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert [res[r][0] for r in range(world)] == [11.0, 11.0]  # max over ranks
    assert res[0][1] != res[1][1]  # each rank has its own batch
