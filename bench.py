"""Benchmark: implied volatilities per second on the 16,777,216-quote BSM grid.

One step = one pass of the whole implied-volatility path (validation,
normalisation, status, intrinsic reduction, LBR boundaries, four-region guess,
Householder(3) steps, store) over the 4,096 strikes x 4,096 maturities grid,
on inputs resident in HBM (822 MB, larger than the 129 MB L2, so no flush is
needed between steps).  `value` is quotes per second over all ranks (each rank
solves its own grid: weak scaling, no collective on the data path).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fv|reference]
                       [--path lbr|mixed|fp32|halley] [--strikes S --maturities M]
Under torchrun (N > 1) every rank runs its own grid; rank 0 prints one JSON line.
`--impl reference` times the CPU oracle on bounded samples of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2604_27210_gb300 import workloads as wl  # noqa: E402

METRIC = "IVs/sec on 16M-quote chain: FP64 LBR vs mixed FP32+FP64, % HBM roofline"
UNIT = "IV/s"
# algorithmic HBM bytes per quote: P, S, K, T, r, q (8 B each) + flag (1 B) in,
# sigma (8 B) + status (1 B) out
BYTES_PER_QUOTE = 58
# The method's FP64 work per quote on this workload, from the counted build of
# the oracle's FP64 LBR (oracle/count_ops.py, a seeded sample of 131,072
# quotes of the grid, written to oracle/op_counts.json): the status rule, two
# Householder(3) iterations (Section 2.2: two suffice) and sigma = s/sqrt(T),
# every +, -, *, /, square root counted and each elementary function at a
# nominal FP64 cost.  The mixed path's FP64 work is the status rule, one
# Householder(3) correction and sigma; the FP32 path's the status rule and
# sigma.  A fixed figure per quote: a faster kernel raises the fraction.
ALG_FLOPS_PER_QUOTE = {"lbr": 370.4, "mixed": 237.4, "fp32": 85.7}
# FP64 flops per quote the step's kernels execute on this workload (DADD +
# DMUL + 2 x DFMA thread-level ncu counters on 4,194,304 quotes of the grid:
# the solver, plus 4.2 per quote in the refinement pass over the quotes it
# marked; profiles/iv_lbr_bsm_grid_4m.md, profiles/kernels_counters_4m.md),
# shown beside the algorithmic figure.
EXECUTED_FLOPS_PER_QUOTE = {"lbr": 307.2 + 4.2}
# The mixed and FP32 solvers run their status rule, reduction and correction in
# double-float arithmetic on the FP32 pipe (1.6 FP64 flops per quote remain):
# their roofline is the FP32 pipe, with the FP32 flops (FADD + FMUL + 2 x FFMA)
# the same captures count per quote, against the measured FFMA rate.
EXECUTED_FP32_FLOPS_PER_QUOTE = {"mixed": 1940.3, "fp32": 1298.0}
FP32_PEAK_GFLOPS = 2 * 37459.7  # 37.46 T FFMA/s, bench_fp64_probe.py
# DRAM bytes (read + write) per quote of the step's kernels from one ncu
# capture each (dram__bytes_read.sum + dram__bytes_write.sum) on 4,194,304
# quotes of the grid (profiles/iv_lbr_bsm_grid_4m.md): the solver, then the
# refinement pass (13.70 MB: the status bytes and the marked quotes' inputs;
# the same scan and the same marked quotes in both precisions).  Traffic grows
# in proportion to the quotes, so a step's traffic is this x n.
DRAM_BYTES_PER_QUOTE_NCU = {"lbr": (206.03e6 + 25.57e6 + 13.70e6) / 4194304,
                            "mixed": (206.31e6 + 26.39e6 + 13.70e6) / 4194304}
# FP64 peaks: measured on this machine's GB300 by bench_fp64_probe.py (526 G
# DFMA/s = 1,052 GFLOP/s; profiles/fp64_fp32_throughput_probe.md), and the
# unit-count figure 152 SMs x 2 FP64 FMA lanes per clock x 2 flops x 2070 MHz
FP64_PEAK_GFLOPS = 1052.0
FP64_PEAK_NOMINAL_GFLOPS = 152 * 2 * 2 * 2.070
SM_MAX_MHZ = 2070.0


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, world_size):
    """Max of a float over all ranks (identity for one rank)."""
    if world_size <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(quotes_per_rank, ms_per_step_local, world_size):
    """Whole-job throughput: every rank solves its own quotes, the job's step
    time is the slowest rank's.  Returns (ms_per_step_max, quotes_per_second)."""
    ms = max_over_ranks(ms_per_step_local, world_size)
    return ms, world_size * quotes_per_rank / (ms * 1e-3)


def barrier(world_size):
    if world_size > 1:
        import torch.distributed as dist
        dist.barrier()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
            os.unlink(self.path)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        # "under load": samples within the top half of the observed clock range
        load = [v for v in sm if v >= 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def make_inputs(fv, torch, dev, n_strikes, n_maturities, seed):
    """The BSM grid on the device, priced by the library's own pricing kernel."""
    w = wl.bsm_grid(n_strikes, n_maturities, seed=seed)
    t = {k: torch.from_numpy(np.ascontiguousarray(w[k])).to(dev) for k in
         ("S_or_F", "K", "T", "r", "q", "flag")}
    mask = torch.from_numpy(w["below_mask"]).to(dev)
    sig = torch.from_numpy(w["sigma_true"]).to(dev)
    sig = torch.where(mask, torch.zeros_like(sig), sig)
    P = fv.fv_price(fv.FV_BSM, t["flag"], t["S_or_F"], t["K"], t["T"], t["r"], t["q"], sig)
    P = torch.where(mask, P * torch.from_numpy(w["below_factor"]).to(dev), P)
    t["P"] = P.contiguous()
    torch.cuda.synchronize()
    return t, w


def run_path(fv, t, path, out, st):
    args = (t["P"], t["S_or_F"], t["K"], t["T"], t["r"], t["q"], t["flag"])
    if path == "lbr":
        fv.fv_implied_vol(fv.FV_BSM, fv.FV_LBR, *args, out, st)
    elif path == "halley":
        fv.fv_implied_vol(fv.FV_BSM, fv.FV_HALLEY, *args, out, st)
    elif path == "mixed":
        fv.fv_implied_vol_ex(fv.FV_BSM, fv.FV_LBR, fv.FV_MIXED, *args, out, st)
    elif path == "fp32":
        fv.fv_implied_vol_ex(fv.FV_BSM, fv.FV_LBR, fv.FV_FP32, *args, out, st)
    else:
        raise ValueError(path)


# kernels per step on the grid: the LBR solver, then the refinement kernel
# over the ill-conditioned quotes it marked (the FP32 path has none; Halley
# refines inside its one kernel)
LAUNCHES_PER_STEP = {"lbr": 2, "mixed": 2, "fp32": 1, "halley": 1}


def halley_fallback_fraction(fv, torch, t, model=None):
    """Share of the quotes the Halley sweeps hand to the fallback: those that
    fail the convergence test after the eighth sweep, and those the cubic-reach
    test sends on earlier (too far from the root at sweep k to reach the
    tolerance by the eighth).  The workspace arrangement of the same solver
    leaves the length of its compacted fallback list in the first four bytes
    of the workspace."""
    model = fv.FV_BSM if model is None else model
    n = t["P"].numel()
    ws = torch.zeros(fv.fv_workspace_size(fv.FV_HALLEY, n), dtype=torch.uint8, device=t["P"].device)
    fv.fv_implied_vol_ws(model, fv.FV_HALLEY, t["P"], t["S_or_F"], t["K"], t["T"], t["r"],
                         t.get("q"), t["flag"], ws)
    torch.cuda.synchronize()
    return int(ws[:4].cpu().numpy().view(np.uint32)[0]) / n


def time_steps(torch, fn, steps, warmup, world_size):
    """W untimed steps, then K steps between barrier + synchronize; CUDA events
    on the current stream (the stream the library launches on)."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    barrier(world_size)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    per = []
    e0.record(stream)
    for _ in range(steps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        per.append((a, b))
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world_size)
    total_ms = e0.elapsed_time(e1)
    kernel_ms = [a.elapsed_time(b) for a, b in per]
    return total_ms, kernel_ms


def _per_rep_us(torch, fn, reps):
    for _ in range(20):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return 1e3 * e0.elapsed_time(e1) / reps


def _black76_batch(fv, torch, dev, n, seed=0):
    """n Black-76 quotes of the small configuration's distribution (F = 100,
    K = F e^k, k ~ U[-1/2, 1/2], T ~ U[0.02, 2], r = 0.03, alternating flags),
    priced by the library's own pricing kernel."""
    w = wl.black76_quotes(n, seed=seed)
    t = {k: torch.from_numpy(np.ascontiguousarray(w[k])).to(dev) for k in ("S_or_F", "K", "T", "r", "flag")}
    sig = torch.from_numpy(w["sigma_true"]).to(dev)
    t["P"] = fv.fv_price(fv.FV_BLACK76, t["flag"], t["S_or_F"], t["K"], t["T"], t["r"], None, sig)
    return t


def small_batch_latency(fv, torch, dev, reps=200):
    """Latency of the FP64 LBR on the 4,096 Black-76 quotes of the small
    configuration: microseconds per call, and per replay of the call captured
    in a CUDA graph (launch overhead out)."""
    t = _black76_batch(fv, torch, dev, 4096)
    out = torch.empty(4096, dtype=torch.float64, device=dev)
    st = torch.empty(4096, dtype=torch.uint8, device=dev)
    call = lambda: fv.fv_implied_vol(fv.FV_BLACK76, fv.FV_LBR, t["P"], t["S_or_F"], t["K"], t["T"],
                                     t["r"], None, t["flag"], out, st)
    call_us = _per_rep_us(torch, call, reps)
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(g, stream=side):
        call()
    torch.cuda.current_stream().wait_stream(side)
    graph_us = _per_rep_us(torch, g.replay, reps)
    return {"quotes": 4096, "workload": "Black-76 4,096 quotes", "call_us": call_us, "graph_us": graph_us,
            "path": "lbr"}


def paper_batch_latency(fv, torch, dev, n=100000, reps=100):
    """The paper's benchmark batch size (Table 3: N = 10^5 quotes, CUDA events):
    microseconds per call of every solver on n Black-76 quotes of the small
    configuration's distribution (inputs 4.1 MB, L2-resident across the
    back-to-back calls), and the Halley sweeps' hand-off share there."""
    t = _black76_batch(fv, torch, dev, n, seed=5)
    out = torch.empty(n, dtype=torch.float64, device=dev)
    st = torch.empty(n, dtype=torch.uint8, device=dev)
    res = {"quotes": n, "workload": "Black-76 %d quotes, the small configuration's distribution" % n}
    for name, solver, prec in (("lbr", fv.FV_LBR, fv.FV_FP64), ("mixed", fv.FV_LBR, fv.FV_MIXED),
                               ("fp32", fv.FV_LBR, fv.FV_FP32), ("halley", fv.FV_HALLEY, fv.FV_FP64),
                               ("halley32", fv.FV_HALLEY, fv.FV_FP32)):
        call = lambda: fv.fv_implied_vol_ex(fv.FV_BLACK76, solver, prec, t["P"], t["S_or_F"], t["K"],
                                            t["T"], t["r"], None, t["flag"], out, st)
        res[name + "_us"] = _per_rep_us(torch, call, reps)
    res["halley_fallback_fraction"] = halley_fallback_fraction(fv, torch, t, fv.FV_BLACK76)
    return res


E2E_CHUNK = 1 << 20


def e2e_measure(fv, torch, w_host, t_dev, steps, warmup, path, transfer):
    """The same metric through the public API from pinned host buffers: each step
    is one fv_implied_vol_host call.  Its inputs start in host memory and sigma +
    status end there; the timed region holds their whole way across the
    CPU-GPU link.  transfer = FV_TRANSFER_DIRECT: the solver reads the inputs
    and writes the outputs in host memory itself (one launch, no staging);
    FV_TRANSFER_STAGED: 1M-quote chunks copied to the device and back,
    overlapped with the solve on two streams.  Either way every input byte
    crosses the link once per step (h2d) and every output byte once (d2h).
    Returns (ms per step, h2d bytes, d2h bytes, the mode taken)."""
    keys = ("P", "S_or_F", "K", "T", "r", "q", "flag")
    host = {k: t_dev[k].cpu().pin_memory() for k in keys}
    n = t_dev["P"].numel()
    out_h = torch.empty(n, dtype=torch.float64).pin_memory()
    st_h = torch.empty(n, dtype=torch.uint8).pin_memory()
    plan = fv.fv_stream_plan_create(E2E_CHUNK)
    plan.set_transfer(transfer)
    solver = fv.FV_HALLEY if path == "halley" else fv.FV_LBR
    prec = {"lbr": fv.FV_FP64, "halley": fv.FV_FP64, "mixed": fv.FV_MIXED, "fp32": fv.FV_FP32}[path]

    def step():
        plan.implied_vol(fv.FV_BSM, solver, prec, host["P"], host["S_or_F"], host["K"], host["T"],
                         host["r"], host["q"], host["flag"], out_h, st_h)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms = max(e0.elapsed_time(e1), 1e3 * wall) / steps
    h2d = sum(host[k].numel() * host[k].element_size() for k in keys)
    d2h = n * 9
    taken = {fv.FV_TRANSFER_DIRECT: "direct", fv.FV_TRANSFER_STAGED: "staged"}[plan.last_transfer]
    plan.destroy()
    return ms, h2d, d2h, taken


def other_configs(fv, torch, dev, steps=3):
    """The remaining workloads of the benchmark set, timed beside the headline
    (N = 1 only; inputs priced by the library's own pricing kernel):
      - 67,108,864 Black-76 quotes with FP32 inputs (F, K, T, r, price): the
        mixed, FP64 and FP32 paths on the FP32 arrays, and the FP64 path on the
        same quotes widened to FP64;
      - 10,000 option chains (74.0 M quotes, lengths log-uniform in 8..65,536):
        the tuned persistent kernel replayed from its CUDA graph, one flat
        launch over the concatenated quotes, and one launch per chain;
      - 8,388,608 BSM quotes: the FP64 LBR, the IV adjoint and the Greeks.
    Each figure: quotes / mean CUDA-event time per step after one warm-up."""
    import bench_kernels as bk
    res = {}

    def timed(fn, n, k=steps):
        tm, _ = time_steps(torch, fn, k, 1, 1)
        return {"value": n / (tm / k * 1e-3), "unit": "quotes/s", "ms_per_step": tm / k}

    # FP32 inputs: the price of the FP32 values widened to FP64, rounded to FP32
    w = wl.black76_fp32(1 << 26, seed=2)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    t = {k: T(w[k]) for k in ("S_or_F", "K", "T", "r", "flag")}
    P = fv.fv_price(w["model"], t["flag"], t["S_or_F"].double(), t["K"].double(),
                    t["T"].double(), t["r"].double(), None, T(w["sigma_true"]))
    t["P"], t["q"] = P.float(), None
    n = t["P"].numel()
    cfg = {"quotes": n}
    for name, kern in (("mixed", "mixed"), ("fp64", "lbr"), ("fp32", "fp32")):
        cfg[name] = timed(bk.runner(fv, torch, kern, w, t), n)
    t64 = {k: (v.double() if v is not None and v.dtype == torch.float32 else v) for k, v in t.items()}
    del t, P
    cfg["fp64_fp64_inputs"] = timed(bk.runner(fv, torch, "lbr", w, t64), n)
    res["black76_fp32_inputs_67m"] = cfg
    del t64, w
    torch.cuda.empty_cache()

    w, t = bk.make(fv, torch, dev, "chains", 10000, 3)
    n = t["P"].numel()
    cfg = {"chains": 10000, "quotes": n}
    fn, plan, _ = bk.chains_runner(fv, torch, w, t, "graph")
    cfg["persistent_graph"] = timed(fn, n)
    cfg["persistent_graph"]["plan"] = plan.info()
    del fn, plan
    cfg["flat_launch"] = timed(bk.runner(fv, torch, "lbr", w, t), n)
    fn, _, _ = bk.chains_runner(fv, torch, w, t, "separate")
    cfg["launch_per_chain"] = timed(fn, n, 2)
    del fn
    res["chains_10k"] = cfg
    del t, w
    torch.cuda.empty_cache()

    w, t = bk.make(fv, torch, dev, "bsm", 1 << 23, 4)
    n = t["P"].numel()
    res["bsm_8m"] = {"quotes": n,
                     "iv_fp64": timed(bk.runner(fv, torch, "lbr", w, t), n),
                     "adjoint": timed(bk.runner(fv, torch, "adjoint", w, t), n),
                     "greeks": timed(bk.runner(fv, torch, "greeks", w, t), n)}
    del t, w
    torch.cuda.empty_cache()
    return res


def cpu_baseline(w_host, P_host, n_sample, seed=123):
    """The oracle's FP64 LBR (its own FP64 normalised Black, as it stands) on
    the workload (all of it, or a seeded sample of n_sample quotes), all host
    cores.  Returns (IV/s, cores, quotes, seconds, index, sigma, status)."""
    from oracle import oracle as orc
    n = P_host.size
    if n_sample >= n:
        idx = np.arange(n)
    else:
        idx = np.sort(np.random.default_rng(seed).choice(n, size=n_sample, replace=False))
    sub = {k: np.ascontiguousarray(np.asarray(w_host[k])[idx]) for k in
           ("S_or_F", "K", "T", "r", "q", "flag")}
    P = np.ascontiguousarray(P_host[idx])
    cores = orc.num_threads()
    t0 = time.perf_counter()
    sig, st, _ = orc.iv_lbr_f64(orc.BSM, P, sub["S_or_F"], sub["K"], sub["T"], sub["r"], sub["q"],
                                sub["flag"], n_iter=3, nthreads=cores)
    dt = time.perf_counter() - t0
    return idx.size / dt, cores, idx.size, dt, idx, sig, st


def error_stats(w_host, P_host, idx, sig_gpu, st_gpu, sig_cpu, st_cpu):
    """The timed GPU path against the oracle's FP64 LBR on the same quotes:
    status agreement and the relative sigma difference where the normalised
    vega b' exceeds 1e-8 (x and beta from the oracle's FP64 status rule)."""
    from oracle import oracle as orc
    sub = {k: np.asarray(w_host[k])[idx] for k in ("S_or_F", "K", "T", "r", "q", "flag")}
    _, x, beta, _ = orc.status(orc.BSM, P_host[idx], sub["S_or_F"], sub["K"], sub["T"], sub["r"],
                               sub["q"], sub["flag"])
    g, c = sig_gpu[idx], sig_cpu
    solved = (st_cpu == 0) & (c > 0) & (st_gpu[idx] == 0)
    s = c[solved] * np.sqrt(sub["T"][solved])
    h, t = -np.abs(x[solved]) / s, 0.5 * s
    v = np.exp(-0.5 * (h * h + t * t)) / np.sqrt(2 * np.pi)
    rel = np.abs(g[solved] - c[solved]) / c[solved]
    gate = v > 1e-8
    return {"quotes": int(idx.size), "status_agree": float(np.mean(st_gpu[idx] == st_cpu)),
            "rel_diff_p50": float(np.median(rel[gate])) if gate.any() else None,
            "rel_diff_p99_99": float(np.quantile(rel[gate], 0.9999)) if gate.any() else None,
            "rel_diff_max": float(rel[gate].max()) if gate.any() else None,
            "gate": "normalised vega > 1e-8", "against": "oracle FP64 LBR"}


def reference_arm(args):
    """CPU oracle arm: each step inverts the grid (or a seeded sample of
    --ref-sample quotes of it) with the oracle's FP64 LBR on all host cores."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from oracle import oracle as orc
    n_s, n_m = args.strikes, args.maturities
    w = wl.bsm_grid(n_s, n_m, seed=1)
    n = w["K"].size
    sample = n if args.ref_sample <= 0 else min(args.ref_sample, n)
    g = np.random.default_rng(7)
    cores = orc.num_threads()
    keys = ("S_or_F", "K", "T", "r", "q", "flag", "sigma_true", "below_mask", "below_factor")
    full = None
    if sample == n:
        full = {key: np.asarray(w[key]) for key in keys}
        full["model"] = wl.BSM
        wl.fill_prices(full, orc.price_f64)
    times = []
    for k in range(args.warmup + args.steps):
        if full is not None:
            sub = full
        else:
            idx = np.sort(g.choice(n, size=sample, replace=False))
            sub = {key: np.ascontiguousarray(np.asarray(w[key])[idx]) for key in keys}
            sub["model"] = wl.BSM
            wl.fill_prices(sub, orc.price_f64)
        t0 = time.perf_counter()
        orc.iv_lbr_f64(orc.BSM, sub["P"], sub["S_or_F"], sub["K"], sub["T"], sub["r"], sub["q"],
                       sub["flag"], n_iter=3, nthreads=cores)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = sample * len(times) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "BSM grid %d strikes x %d maturities (%d quotes per step)"
                                   % (n_s, n_m, sample),
                       "solver": "LBR (CPU oracle, FP64 steps and FP64 normalised Black)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": ("the whole grid per step" if sample == n else
                                        "%d seeded quotes of the grid per step" % sample)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fv", choices=["fv", "reference"])
    ap.add_argument("--path", default="lbr", choices=["lbr", "mixed", "fp32", "halley"])
    ap.add_argument("--strikes", type=int, default=4096)
    ap.add_argument("--maturities", type=int, default=4096)
    ap.add_argument("--ref-sample", type=int, default=0, help="quotes per reference step (0: all)")
    ap.add_argument("--cpu-sample", type=int, default=1 << 30, help="quotes of the CPU baseline")
    ap.add_argument("--no-extras", action="store_true",
                    help="time only the selected path (for profiler runs)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other workloads (FP32 inputs, chains, BSM adjoint)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)

    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_2604_27210_gb300 import fv

    t, w = make_inputs(fv, torch, dev, args.strikes, args.maturities, seed=1 + rank)
    n = t["P"].numel()
    out = torch.empty(n, dtype=torch.float64, device=dev)
    st = torch.empty(n, dtype=torch.uint8, device=dev)

    with ClockSampler(local if ws > 1 else 0) as clk:
        total_ms, kernel_ms = time_steps(torch, lambda: run_path(fv, t, args.path, out, st),
                                         args.steps, args.warmup, ws)
    clocks = clk.summary()
    ms_step, value = aggregate(n, total_ms / args.steps, ws)

    # roofline of the step's kernels: the solver (97 % of the step's device
    # time on the grid) and its refinement pass
    k_ms = statistics.mean(kernel_ms)
    hbm_peak, hbm_kind = peaks()
    gbs = BYTES_PER_QUOTE * n / (k_ms * 1e-3) / 1e9
    flops_q = ALG_FLOPS_PER_QUOTE.get(args.path)
    if args.path in EXECUTED_FP32_FLOPS_PER_QUOTE:
        f32_q = EXECUTED_FP32_FLOPS_PER_QUOTE[args.path]
        achieved = f32_q * n / (k_ms * 1e-3) / 1e9
        dram_q = DRAM_BYTES_PER_QUOTE_NCU.get(args.path)
        roofline = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_GFLOPS,
                    "unit": "GFLOP/s (FP32)", "frac": achieved / FP32_PEAK_GFLOPS,
                    "traffic": dram_q * n if dram_q is not None else None,
                    "flops_per_quote": f32_q,
                    "flops_kind": "executed: FP32 flops per quote of the solver (ncu); the kernel is "
                                  "bound by instruction issue, not by the FP32 pipe",
                    "fp64_method_flops_per_quote": flops_q,
                    "peak_kind": "measured FP32 FMA rate on this GPU (bench_fp64_probe.py)"}
    elif flops_q is not None:
        achieved = flops_q * n / (k_ms * 1e-3) / 1e9
        dram_q = DRAM_BYTES_PER_QUOTE_NCU.get(args.path)
        roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GFLOPS,
                    "unit": "GFLOP/s (FP64)", "frac": achieved / FP64_PEAK_GFLOPS,
                    "traffic": dram_q * n if dram_q is not None else None,
                    "flops_per_quote": flops_q,
                    "flops_kind": "algorithmic: the method's FP64 operations per quote from the "
                                  "counted build of the oracle's FP64 LBR (oracle/count_ops.py)",
                    "executed_flops_per_quote": EXECUTED_FLOPS_PER_QUOTE.get(args.path),
                    "peak_kind": "measured FP64 FMA rate on this GPU (bench_fp64_probe.py)",
                    "peak_nominal": FP64_PEAK_NOMINAL_GFLOPS,
                    "frac_of_nominal": achieved / FP64_PEAK_NOMINAL_GFLOPS}
    else:
        roofline = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                    "frac": gbs / hbm_peak, "traffic": None}
    hbm = {"achieved_gbs": gbs, "peak_gbs": hbm_peak, "peak_kind": hbm_kind,
           "frac": gbs / hbm_peak, "bytes_per_quote": BYTES_PER_QUOTE}

    extras = {}
    if not args.no_extras:
        for p, k in (("mixed", args.steps), ("fp32", args.steps), ("halley", 3)):
            if p == args.path:
                continue
            tm, km = time_steps(torch, lambda: run_path(fv, t, p, out, st), k, 1, ws)
            extras[p] = {"value": ws * n / (max_over_ranks(tm / k, ws) * 1e-3),
                         "ms_per_step": tm / k,
                         "hbm_frac": BYTES_PER_QUOTE * n / (statistics.mean(km) * 1e-3) / 1e9 / hbm_peak}
        extras.setdefault("halley", {})["fallback_fraction"] = halley_fallback_fraction(fv, torch, t)
        extras["small_batch"] = small_batch_latency(fv, torch, dev)
        extras["paper_batch"] = paper_batch_latency(fv, torch, dev)
        # pricing and Greeks on the same grid
        sig = t["P"].new_tensor(w["sigma_true"])
        for name, fn in (("price", lambda: fv.fv_price(fv.FV_BSM, t["flag"], t["S_or_F"], t["K"],
                                                        t["T"], t["r"], t["q"], sig, out)),
                         ("greeks", lambda: fv.fv_greeks(fv.FV_BSM, t["flag"], t["S_or_F"], t["K"],
                                                          t["T"], t["r"], t["q"], sig))):
            tm, _ = time_steps(torch, fn, 5, 1, ws)
            extras[name] = {"value": ws * n / (max_over_ranks(tm / 5, ws) * 1e-3), "unit": "quotes/s",
                            "ms_per_step": tm / 5}

    e2e_steps = max(3, args.steps // 4)
    e2e_ms, h2d, d2h, e2e_mode = e2e_measure(fv, torch, w, t, e2e_steps, 1, args.path,
                                             fv.FV_TRANSFER_AUTO)
    e2e_ms = max_over_ranks(e2e_ms, ws)
    # the chunked-copy pipeline on the same buffers, for comparison
    staged_ms = max_over_ranks(e2e_measure(fv, torch, w, t, e2e_steps, 1, args.path,
                                           fv.FV_TRANSFER_STAGED)[0], ws)

    cpu = None
    errors = None
    if rank == 0 and ws == 1:
        P_host = t["P"].cpu().numpy()
        rate, cores, m, dt, idx, sig_cpu, st_cpu = cpu_baseline(w, P_host, args.cpu_sample)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d quotes of the grid (%s), oracle FP64 LBR (3 Householder steps, its own "
                         "FP64 normalised Black), %.1f s" % (m, "all" if m == n else "seeded sample",
                                                              dt)}
        # the timed path's outputs of its last step against the CPU solver
        run_path(fv, t, args.path, out, st)
        torch.cuda.synchronize()
        errors = error_stats(w, P_host, idx, out.cpu().numpy(), st.cpu().numpy(), sig_cpu, st_cpu)

    configs = None
    if ws == 1 and not args.no_extras and not args.no_configs:
        del t, out, st
        torch.cuda.empty_cache()
        configs = other_configs(fv, torch, dev)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.path in ("lbr", "halley") else
                ("f32+f64" if args.path == "mixed" else "f32"),
                "data": "synthetic",
                "config": {"workload": "BSM grid %d strikes x %d maturities = %d quotes per GPU, "
                                       "S=100, log-moneyness [-3,3], T log-spaced [1/365,5], "
                                       "r~U[0,.06], q~U[0,.05], sigma~U[.01,3], 5%% below intrinsic"
                                       % (args.strikes, args.maturities, n),
                           "path": args.path, "solver": "LBR" if args.path != "halley" else "Halley",
                           "inputs_vs_l2": "inputs %.0f MB > 129 MB L2: no flush between steps"
                                           % (n * 49 / 1e6),
                           "parallelism": "replicas x%d (one grid per GPU)" % ws},
                "roofline": roofline, "hbm_roofline": hbm,
                "clocks": clocks, "gpu_launches": LAUNCHES_PER_STEP[args.path] * args.steps,
                "e2e": {"value": ws * n / (e2e_ms * 1e-3), "unit": UNIT,
                        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                        "ms_per_step": e2e_ms, "transfer": e2e_mode,
                        "staged_value": ws * n / (staged_ms * 1e-3)},
                "cpu_baseline": cpu, "errors": errors, "paths": extras, "configs": configs}
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
