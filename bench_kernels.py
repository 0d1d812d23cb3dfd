"""Per-kernel timing driver: one entry point of libfv.so on one synthetic workload.

Used for profiler captures of a single kernel and for throughput-versus-N
sweeps.  Prints one JSON line per size:

  python bench_kernels.py --kernel lbr --workload grid \
      --n 4194304 --reps 5 --warmup 2

kernels:   lbr, mixed, fp32, halley, halley32, price, greeks, adjoint, chains
workloads: grid (BSM strike x maturity grid), b76 (Black-76 quotes),
           b76f32 (the same in FP32), bsm (BSM quotes with an upstream
           gradient), chains (option chains; --n is the number of chains)
Inputs are priced by the library's own pricing kernel.  --graph captures
the call once in a CUDA graph and times its replays (launch overhead out).
"""
import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2604_27210_gb300 import workloads as wl  # noqa: E402


def _grid_dims(n):
    ns = 4096 if n >= 4096 else n
    return ns, max(1, n // ns)


def make(fv, torch, dev, workload, n, seed):
    if workload == "grid":
        ns, nm = _grid_dims(n)
        w = wl.bsm_grid(ns, nm, seed=seed)
    elif workload in ("b76", "b76f32"):
        w = wl.black76_quotes(n, seed=seed)
    elif workload == "bsm":
        w = wl.bsm_quotes(n, seed=seed)
    elif workload == "chains":
        w = wl.chains(n, seed=seed)
    else:
        raise ValueError(workload)
    T = lambda a, dt=None: torch.from_numpy(np.ascontiguousarray(a if dt is None else a.astype(dt))).to(dev)
    t = {k: T(w[k]) for k in ("S_or_F", "K", "T", "r", "flag") if w.get(k) is not None}
    t["q"] = T(w["q"]) if w.get("q") is not None else None
    sig = T(w["sigma_true"])
    if w.get("below_mask") is not None:
        mask = T(w["below_mask"])
        sig0 = torch.where(mask, torch.zeros_like(sig), sig)
    else:
        mask, sig0 = None, sig
    P = fv.fv_price(w["model"], t["flag"], t["S_or_F"], t["K"], t["T"], t["r"], t["q"], sig0)
    if mask is not None:
        P = torch.where(mask, P * T(w["below_factor"]), P)
    t["P"] = P.contiguous()
    t["sigma_true"] = sig
    if w.get("grad_sigma") is not None:
        t["grad_sigma"] = T(w["grad_sigma"])
    if workload == "b76f32":
        for k in ("P", "S_or_F", "K", "T", "r"):
            t[k] = t[k].float()
    return w, t


def runner(fv, torch, kernel, w, t):
    model = w["model"]
    n = t["P"].numel()
    dev = t["P"].device
    out = torch.empty(n, dtype=torch.float64, device=dev)
    st = torch.empty(n, dtype=torch.uint8, device=dev)
    a = (t["P"], t["S_or_F"], t["K"], t["T"], t["r"], t["q"], t["flag"])
    if kernel == "lbr":
        if t["P"].dtype == torch.float32:
            return lambda: fv.fv_implied_vol_ex(model, fv.FV_LBR, fv.FV_FP64, *a, out, st)
        return lambda: fv.fv_implied_vol(model, fv.FV_LBR, *a, out, st)
    if kernel == "halley":
        return lambda: fv.fv_implied_vol(model, fv.FV_HALLEY, *a, out, st)
    if kernel == "halley32":
        return lambda: fv.fv_implied_vol_ex(model, fv.FV_HALLEY, fv.FV_FP32, *a, out, st)
    if kernel == "mixed":
        return lambda: fv.fv_implied_vol_ex(model, fv.FV_LBR, fv.FV_MIXED, *a, out, st)
    if kernel == "fp32":
        return lambda: fv.fv_implied_vol_ex(model, fv.FV_LBR, fv.FV_FP32, *a, out, st)
    if kernel == "price":
        return lambda: fv.fv_price(model, t["flag"], t["S_or_F"], t["K"], t["T"], t["r"], t["q"],
                                   t["sigma_true"], out)
    if kernel == "greeks":
        return lambda: fv.fv_greeks(model, t["flag"], t["S_or_F"], t["K"], t["T"], t["r"], t["q"],
                                    t["sigma_true"])
    if kernel == "adjoint":
        fv.fv_implied_vol(model, fv.FV_LBR, *a, out, st)
        g = t.get("grad_sigma", torch.ones(n, dtype=torch.float64, device=dev))
        return lambda: fv.fv_iv_adjoint(model, *a, out, st, g)
    raise ValueError(kernel)


def chains_runner(fv, torch, w, t, mode):
    dev = t["P"].device
    off = w["offsets"]
    chains = []
    for j in range(len(w["lens"])):
        a, b = int(off[j]), int(off[j + 1])
        chains.append(dict(price=t["P"][a:b].contiguous(), K=t["K"][a:b].contiguous(),
                           flag=t["flag"][a:b].contiguous(),
                           sigma=torch.empty(b - a, dtype=torch.float64, device=dev),
                           status=torch.empty(b - a, dtype=torch.uint8, device=dev),
                           S_or_F=w["F_chain"][j], T=w["T_chain"][j], r=w["r_chain"][j]))
    if mode == "separate":
        # one ordinary launch per chain (per-chain F, T, r broadcast to arrays once)
        for c in chains:
            n = c["price"].numel()
            for k in ("S_or_F", "T", "r"):
                c[k + "_arr"] = torch.full((n,), c[k], dtype=torch.float64, device=dev)

        def run():
            for c in chains:
                fv.fv_implied_vol(fv.FV_BLACK76, fv.FV_LBR, c["price"], c["S_or_F_arr"], c["K"],
                                  c["T_arr"], c["r_arr"], None, c["flag"], c["sigma"], c["status"])
        return run, None, chains
    plan = fv.fv_chains_plan_create(fv.FV_BLACK76, chains, autotune=(mode == "graph"))
    return (plan.run if mode == "graph" else plan.run_direct), plan, chains


def time_it(torch, fn, reps, warmup, graph=False):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if graph:
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                fn()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        fn = g.replay
        fn()
        torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kernel", default="lbr")
    ap.add_argument("--workload", default="grid")
    ap.add_argument("--n", type=int, nargs="+", default=[1 << 22])
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--chains-mode", default="graph", choices=["graph", "direct", "separate", "flat"])
    ap.add_argument("--graph", action="store_true", help="time CUDA-graph replays of the call")
    args = ap.parse_args()
    import torch
    from paper_2604_27210_gb300 import fv
    dev = torch.device("cuda:0")
    for n in args.n:
        w, t = make(fv, torch, dev, args.workload, n, args.seed)
        quotes = t["P"].numel()
        extra = {}
        if args.kernel == "chains":
            if args.chains_mode == "flat":
                fn = runner(fv, torch, "lbr", w, t)
            else:
                fn, plan, _ = chains_runner(fv, torch, w, t, args.chains_mode)
                if plan is not None:
                    extra["plan"] = plan.info()
        else:
            fn = runner(fv, torch, args.kernel, w, t)
        ms = time_it(torch, fn, args.reps, args.warmup, graph=args.graph and args.kernel != "chains")
        line = {"kernel": args.kernel, "workload": args.workload, "n": n, "quotes": quotes,
                "ms": ms, "quotes_per_s": quotes / (ms * 1e-3)}
        line.update(extra)
        if args.kernel == "chains":
            line["chains_mode"] = args.chains_mode
        if args.graph and args.kernel != "chains":
            line["graph"] = True
        print(json.dumps(line), flush=True)
        del t, fn
        torch.cuda.empty_cache()


if __name__ == "__main__":
    main()
