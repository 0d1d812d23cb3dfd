"""The benchmark's multi-rank path on the CPU: two gloo ranks, each with its own
quotes and its own step time, aggregate to the slowest rank's time and the
whole job's quote count (weak scaling, no collective on the data path)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench._dist()
        assert (ws, r, local) == (world, rank, rank)
        bench.barrier(ws)
        ms, value = bench.aggregate(1000, 10.0 + 5.0 * rank, ws)
        q.put((rank, ms, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_to_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in res:
        assert ms == pytest.approx(15.0)
        assert value == pytest.approx(2 * 1000 / 15e-3)


def test_single_rank_is_identity():
    import bench
    ms, value = bench.aggregate(500, 4.0, 1)
    assert ms == 4.0 and value == pytest.approx(500 / 4e-3)
