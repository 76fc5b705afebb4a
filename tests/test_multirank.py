"""The N > 1 host logic of bench.py (replicas: barrier, max-over-ranks timing, whole-job
throughput) on CPU with the gloo backend, world size 2."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        secs = [1.5, 2.25][rank]
        elems = [1000, 3000][rank]
        dist.barrier()
        mx = bench.max_over_ranks(secs, "cpu")
        tot = bench.sum_over_ranks(elems, "cpu")
        q.put((rank, mx, tot, bench.aggregate([tot], [mx]), bench._dist()))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, tot, val, d in res:
        assert mx == 2.25 and tot == 4000
        assert val == pytest.approx(4000 / 2.25)
        assert d == (rank, 2, rank)


def test_single_process_passthrough():
    import bench
    assert bench.max_over_ranks(3.0, "cpu") == 3.0
    assert bench.aggregate([10, 20], [1.0, 2.0]) == 15.0
