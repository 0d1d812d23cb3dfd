"""One batch over several GPUs: the partitions (CPU), the gather of the
shards' outputs over two gloo ranks (CPU), and the shards solved one after
another on one GPU against the whole batch (gpu)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2604_27210_gb300 import shard
from paper_2604_27210_gb300 import workloads as wl


@pytest.mark.parametrize("n,world", [(0, 1), (1, 2), (7, 3), (16777216, 8), (1000003, 4)])
def test_quote_ranges_partition_the_batch(n, world):
    rs = [shard.quote_range(n, k, world) for k in range(world)]
    assert rs[0][0] == 0 and rs[-1][1] == n
    assert all(rs[k][1] == rs[k + 1][0] for k in range(world - 1))
    sizes = [b - a for a, b in rs]
    assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("world", [1, 2, 4, 8])
def test_chain_shards_balance_whole_chains(world):
    lens = wl.chains(10000, seed=3)["lens"]
    sh = shard.chain_shards(lens, world)
    flat = np.concatenate([np.asarray(s, dtype=np.int64) for s in sh])
    assert np.array_equal(np.sort(flat), np.arange(lens.size))  # every chain once
    loads = np.array([lens[s].sum() for s in sh])
    assert loads.sum() == lens.sum()
    # LPT: the largest load exceeds the mean by at most one chain, and here by
    # far less than one per cent
    assert loads.max() <= lens.sum() / world + lens.max()
    assert loads.max() <= 1.01 * lens.sum() / world


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        a, b = shard.quote_range(n, rank, world)
        sigma = torch.arange(a, b, dtype=torch.float64) * 0.5  # a stand-in for the shard's solve
        status = (torch.arange(a, b) % 4).to(torch.uint8)
        s_all, t_all = shard.gather_shards(sigma, status, n, rank, world)
        q.put((rank, bool(torch.equal(s_all, torch.arange(n, dtype=torch.float64) * 0.5)),
               bool(torch.equal(t_all, (torch.arange(n) % 4).to(torch.uint8)))))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_gather_their_shards():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, 1001, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert res == [(0, True, True), (1, True, True)]


@pytest.mark.gpu
def test_shards_solved_in_turn_equal_the_whole_batch():
    # each rank's range through the library (here one after another on one GPU)
    import torch
    from oracle import oracle as orc
    from paper_2604_27210_gb300 import fv
    dev = torch.device("cuda:0")
    w = wl.fill_prices(wl.bsm_grid(1000, 300, seed=47), orc.price_f64)
    t = {k: torch.tensor(np.ascontiguousarray(w[k]), device=dev)
         for k in ("P", "S_or_F", "K", "T", "r", "q", "flag")}
    args = [t[k] for k in ("P", "S_or_F", "K", "T", "r", "q", "flag")]
    s_all, st_all = fv.fv_implied_vol_ex(fv.FV_BSM, fv.FV_LBR, fv.FV_FP64, *args)
    parts = [shard.implied_vol_shard(fv, fv.FV_BSM, fv.FV_LBR, fv.FV_FP64, *args, rank, 3)
             for rank in range(3)]
    assert [p[0] for p in parts] == [shard.quote_range(t["P"].numel(), k, 3)[0] for k in range(3)]
    s = torch.cat([p[2] for p in parts])
    st = torch.cat([p[3] for p in parts])
    assert torch.equal(st, st_all)
    ok = ~torch.isnan(s_all) & (s_all > 0)
    assert torch.equal(torch.isnan(s), torch.isnan(s_all))
    assert torch.all((s[ok] - s_all[ok]).abs() <= 1e-12 * s_all[ok])
