"""Count the FP64 work of the implied-volatility method per quote (oracle tooling).

Builds the counted build of the oracle's FP64 LBR (op_count.cpp over
lbr_steps.h) and runs it over seeded samples of the five workloads: the FP64
status rule, then, for the quotes that need a root, the LBR steps of Section
2.2 with three Householder(3) iterations (the oracle's FP64 solver).  Every
+, -, *, /, square root and fused multiply-add is counted, and every
elementary-function call; the calls are converted to FP64 operations with
the nominal costs of COSTS (textbook table-driven or polynomial
implementations at FP64 accuracy), so that the method's work per quote is one
number that no implementation detail of the kernels changes.

    python oracle/count_ops.py            # prints the table, writes oracle/op_counts.json

Only the tests and this script run the counted build; the library and the
benchmark never do (the benchmark quotes the grid's figure as a constant).
"""
import ctypes
import json
import os
import subprocess
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import oracle as orc  # noqa: E402
from paper_2604_27210_gb300 import workloads as wl  # noqa: E402

LIB = os.path.join(HERE, "_build", "liboc.so")
OUT = os.path.join(HERE, "op_counts.json")
FIELDS = ["add", "mul", "div", "sqrt", "fma", "cmp", "exp", "expm1", "log", "log1p", "erfc",
          "erfcx", "cbrt", "sinh", "ncdfinv"]
# FP64 operations per counted item.  Additions, multiplications, divisions and
# square roots are IEEE basic operations (1 each), a fused multiply-add is 2,
# comparisons are not arithmetic (0).  Elementary functions at FP64 accuracy:
# exp / expm1 / sinh by a table-driven reduction and a degree-5 polynomial (15),
# log / log1p by a table-driven reduction and a degree-6 polynomial (20),
# erfcx by a piecewise degree-8 polynomial on a located interval (20), erfc as
# erfcx times exp(-z^2) (35), cbrt by a polynomial seed and two Newton steps
# (15), the inverse normal CDF by a rational approximation of two degree-7
# polynomials (30).
COSTS = {"add": 1, "mul": 1, "div": 1, "sqrt": 1, "fma": 2, "cmp": 0, "exp": 15, "expm1": 15,
         "log": 20, "log1p": 20, "erfc": 35, "erfcx": 20, "cbrt": 15, "sinh": 15, "ncdfinv": 30}
REGIONS = {-1: "no root", 0: "lowest", 1: "lower middle", 2: "upper middle", 3: "highest"}


def build(force=False):
    src = [os.path.join(HERE, f) for f in ("op_count.cpp", "lbr_steps.h", "fv_oracle.h")]
    if not force and os.path.exists(LIB) and all(os.path.getmtime(f) <= os.path.getmtime(LIB)
                                                 for f in src):
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                    "-shared", "-o", tmp, src[0]], check=True)
    os.replace(tmp, LIB)
    return LIB


def count(model, w, n_iter=3):
    """Per-quote cumulative counts (n x (n_iter + 3) x len(FIELDS) int64: after the
    status rule, after the boundaries and guess, after each iteration, at the
    end), regions and sigma."""
    lib = ctypes.CDLL(build())
    assert lib.oc_num_counts() == len(FIELDS)
    D = ctypes.POINTER(ctypes.c_double)
    n = np.asarray(w["K"]).size
    f = lambda k: np.ascontiguousarray(np.broadcast_to(np.asarray(
        0.0 if w.get(k) is None else w[k], dtype=np.float64), (n,)))
    ins = [f(k) for k in ("P", "S_or_F", "K", "T", "r", "q")]
    flag = np.ascontiguousarray(w["flag"], dtype=np.int8)
    counts = np.zeros((n, n_iter + 3, len(FIELDS)), np.int64)
    reg = np.zeros(n, np.int8)
    sig = np.zeros(n, np.float64)
    lib.oc_count_lbr.argtypes = [ctypes.c_int] + [D] * 6 + [ctypes.POINTER(ctypes.c_int8),
                                                            ctypes.c_int64, ctypes.c_int,
                                                            ctypes.POINTER(ctypes.c_int64),
                                                            ctypes.POINTER(ctypes.c_int8), D]
    lib.oc_count_lbr(model, *[a.ctypes.data_as(D) for a in ins],
                     flag.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), n, n_iter,
                     counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                     reg.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), sig.ctypes.data_as(D))
    return counts, reg, sig


def flops(counts):
    """FP64 operations (nominal costs for the calls) of counts along the last axis."""
    return counts @ np.array([COSTS[k] for k in FIELDS], dtype=np.int64)


def summarise(model, w, n_iter=3):
    """Mean FP64 operations per quote of the whole oracle solver and of its
    phases, and the method's FP64 work: the status rule, two Householder(3)
    iterations (Section 2.2: two suffice) and sigma = s / sqrt(T).  The
    boundaries and the initial guess only seed the iterations (the guess is
    ~1e-2 off), so the method needs no FP64 for them."""
    counts, reg, sig = count(model, w, n_iter)
    cum = flops(counts)                      # n x (n_iter + 3)
    status = cum[:, 0]
    guess = cum[:, 1] - cum[:, 0]
    iters = np.diff(cum[:, 1:n_iter + 2], axis=1)  # n x n_iter
    final = cum[:, -1] - cum[:, n_iter + 1]
    method = status + iters[:, :2].sum(axis=1) + final
    solving = reg >= 0
    # the FP64 work of each precision path: FP64 LBR (two iterations), mixed
    # (one FP64 correction), FP32 (the status rule and sigma only)
    paths = {"lbr": float(method.mean()), "mixed": float((status + iters[:, 0] + final).mean()),
             "fp32": float((status + final).mean())}
    out = {"quotes": int(cum.shape[0]), "flops_per_quote": float(cum[:, -1].mean()),
           "method_flops_per_quote": float(method.mean()), "method_flops_per_quote_by_path": paths,
           "phases_per_quote": {"status": float(status.mean()), "boundaries_and_guess": float(guess.mean()),
                                "iterations": [float(iters[:, k].mean()) for k in range(n_iter)],
                                "sigma": float(final.mean())},
           "per_solved_quote": {"boundaries_and_guess": float(guess[solving].mean()),
                                "iteration": float(iters[solving][:, :2].mean())} if solving.any() else {},
           "per_quote": {k: float(counts[:, -1, j].mean()) for j, k in enumerate(FIELDS)},
           "by_region": {}}
    for r, name in REGIONS.items():
        m = reg == r
        if m.any():
            out["by_region"][name] = {"fraction": float(m.mean()), "flops_per_quote": float(cum[m, -1].mean()),
                                      "method_flops_per_quote": float(method[m].mean())}
    return out, sig


def workloads(sample=131072, seed=5):
    """Seeded samples of the five workloads, priced by the oracle."""
    g = np.random.default_rng(seed)

    def take(w, n):
        m = np.asarray(w["K"]).size
        idx = np.sort(g.choice(m, size=min(n, m), replace=False))
        sub = {k: (np.asarray(v)[idx] if isinstance(v, np.ndarray) and v.size == m else v)
               for k, v in w.items()}
        return sub

    grid = take(wl.bsm_grid(4096, 4096, seed=1), sample)
    chains = wl.chains(400, seed=3)
    for k in ("lens", "offsets", "F_chain", "T_chain", "r_chain"):
        chains.pop(k)
    f32 = wl.black76_fp32(sample // 4, seed=2)
    for k in ("S_or_F", "K", "T", "r"):
        f32[k] = f32[k].astype(np.float64)
    return [("BSM grid 4096 x 4096 (16,777,216 quotes)", wl.fill_prices(grid, orc.price)),
            ("Black-76 4,096 quotes", wl.fill_prices(wl.black76_quotes(4096, seed=0), orc.price)),
            ("Black-76 FP32 inputs (67,108,864 quotes)", wl.fill_prices(f32, orc.price)),
            ("10,000 chains (74.0 M quotes)", wl.fill_prices(take(chains, sample // 4), orc.price)),
            ("BSM 8,388,608 quotes", wl.fill_prices(wl.bsm_quotes(sample // 4, seed=4), orc.price))]


def main():
    res = {"costs": COSTS, "n_iter": 3, "workloads": {}}
    for name, w in workloads():
        s, sig = summarise(w["model"], w)
        # the counted build runs the oracle's FP64 LBR: the same results
        ref, _, _ = orc.iv_lbr_f64(w["model"], w["P"], w["S_or_F"], w["K"], w["T"], w["r"], w.get("q"),
                                   w["flag"], n_iter=3)
        assert np.array_equal(sig, ref, equal_nan=True), name
        res["workloads"][name] = s
        print("%-42s method %6.1f, oracle solver %6.1f FP64 operations per quote  (%s)" % (
            name, s["method_flops_per_quote"], s["flops_per_quote"],
            ", ".join("%s %.0f%%/%.0f" % (r, 100 * v["fraction"], v["method_flops_per_quote"])
                      for r, v in s["by_region"].items())))
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1, sort_keys=True)
        f.write("\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
