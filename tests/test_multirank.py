"""Host logic of the multi-GPU benchmark on CPU: two gloo ranks on 127.0.0.1.

bench.py --gpus N runs one independent lattice per rank (no collective on the data
path) and reports the units all ranks processed over the slowest rank's timed region.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, l = bench.dist_env()
        ms_local = 100.0 + 50.0 * r  # rank 1 is the slow one
        ms = bench.reduce_max_over_ranks(ms_local, dist, "cpu")
        q.put((r, w, l, ms, bench.job_mlups(2.0e9, w, ms)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert all(r[3] == 150.0 for r in res)  # max over ranks
    # 2 ranks x 2e9 updates in 0.15 s
    assert all(abs(r[4] - 2 * 2.0e9 / 0.15 / 1e6) < 1e-6 for r in res)
