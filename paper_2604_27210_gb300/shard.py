"""One batch over the GPUs of a node: the partition and the optional gather.

Every quote is independent (no collective is needed for the computation), so
a batch splits into one shard per GPU, one process per GPU:
  - quote_range(n, rank, world): a contiguous range of a flat batch, the
    shards' sizes differing by at most one quote;
  - chain_shards(lengths, world): whole option chains per rank, balanced by
    quote count (longest chains first, each to the least-loaded rank: the LPT
    rule, within 4/3 of the best possible maximum load);
  - implied_vol_shard: each rank solves its range of a flat batch on its own
    GPU through the library (no data-path collective);
  - gather_shards: all-gather the shards' sigma and status when a caller wants
    every rank to hold the whole result (NCCL for CUDA tensors, gloo on CPU).
Host-side plumbing only: every quote is solved by the library's kernels.
"""
import heapq

import numpy as np


def quote_range(n, rank, world):
    """[start, stop) of rank's contiguous share of n quotes."""
    if world <= 0 or not 0 <= rank < world or n < 0:
        raise ValueError("need 0 <= rank < world and n >= 0")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def chain_shards(lengths, world):
    """Chain indices per rank (each list ascending): whole chains, the ranks'
    quote counts balanced by the longest-processing-time rule."""
    if world <= 0:
        raise ValueError("world must be positive")
    lengths = np.asarray(lengths, dtype=np.int64)
    order = np.argsort(-lengths, kind="stable")
    heap = [(0, r) for r in range(world)]
    shards = [[] for _ in range(world)]
    for c in order:
        load, r = heapq.heappop(heap)
        shards[r].append(int(c))
        heapq.heappush(heap, (load + int(lengths[c]), r))
    return [sorted(s) for s in shards]


def implied_vol_shard(fv, model, solver, precision, price, S_or_F, K, T, r, q, flag, rank, world):
    """This rank's share of a flat batch: slices [start, stop) of the given
    device tensors (views, no copy) and solves them with fv_implied_vol_ex.
    Returns (start, stop, sigma, status) of the shard."""
    n = price.numel()
    a, b = quote_range(n, rank, world)
    sl = lambda t: None if t is None else t[a:b]
    sigma, status = fv.fv_implied_vol_ex(model, solver, precision, sl(price), sl(S_or_F), sl(K),
                                         sl(T), sl(r), sl(q), sl(flag))
    return a, b, sigma, status


def gather_shards(sigma, status, n, rank, world, group=None):
    """All-gather every rank's contiguous shard (quote_range order) into the
    whole batch's sigma and status on every rank."""
    import torch
    import torch.distributed as dist
    sizes = [quote_range(n, k, world) for k in range(world)]
    m = max(b - a for a, b in sizes)
    pad_s = torch.zeros(m, dtype=sigma.dtype, device=sigma.device)
    pad_t = torch.zeros(m, dtype=status.dtype, device=status.device)
    pad_s[:sigma.numel()] = sigma
    pad_t[:status.numel()] = status
    all_s = [torch.empty_like(pad_s) for _ in range(world)]
    all_t = [torch.empty_like(pad_t) for _ in range(world)]
    dist.all_gather(all_s, pad_s, group=group)
    dist.all_gather(all_t, pad_t, group=group)
    out_s = torch.cat([all_s[k][:b - a] for k, (a, b) in enumerate(sizes)])
    out_t = torch.cat([all_t[k][:b - a] for k, (a, b) in enumerate(sizes)])
    return out_s, out_t
