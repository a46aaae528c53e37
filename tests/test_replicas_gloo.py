"""The replica path of bench.py on two gloo ranks (CPU): each rank solves its own problem,
and the whole-job figure is the units all ranks processed over the slowest rank's time
(replicas only: the sampled solve has no exchange step between GPUs)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        units, secs = [100.0, 50.0][rank], [1.0, 2.0][rank]
        rate, slowest = bench.whole_job_rate(units, secs, world)
        mx = bench.max_over_ranks([3.0, 7.0][rank], world)
        bench.barrier(world)
        q.put((rank, rate, slowest, mx))
    finally:
        dist.destroy_process_group()


def test_whole_job_rate_over_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in procs:
            rank, rate, slowest, mx = q.get(timeout=120)
            out[rank] = (rate, slowest, mx)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    # 150 units in all over the slower rank's 2 s, on every rank
    for r in (0, 1):
        assert out[r] == (75.0, 2.0, 7.0), out


def test_whole_job_rate_single_rank():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.whole_job_rate(120.0, 2.0, 1) == (60.0, 2.0)
    assert bench.max_over_ranks(3.5, 1) == 3.5
