"""The counted build of the oracle's FP64 LBR (oracle/op_count.cpp over
oracle/lbr_steps.h), whose per-quote FP64 operation counts are the numerator
of the benchmark's ALU roofline."""
import json
import os

import numpy as np
import pytest

from oracle import count_ops
from oracle import oracle as orc
from paper_2604_27210_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GRID = "BSM grid 4096 x 4096 (16,777,216 quotes)"


@pytest.fixture(scope="module")
def grid_sample():
    w = wl.bsm_grid(4096, 4096, seed=1)
    idx = np.sort(np.random.default_rng(9).choice(w["K"].size, 16384, replace=False))
    sub = {k: (np.asarray(v)[idx] if isinstance(v, np.ndarray) and v.size == w["K"].size else v)
           for k, v in w.items()}
    return wl.fill_prices(sub, orc.price)


def test_counted_build_runs_the_oracle_solver(grid_sample):
    # same source over the counting scalar: the same sigma, bit for bit
    w = grid_sample
    _, reg, sig = count_ops.count(w["model"], w)
    ref, st, reg_ref = orc.iv_lbr_f64(w["model"], w["P"], w["S_or_F"], w["K"], w["T"], w["r"], w["q"],
                                      w["flag"], n_iter=3)
    assert np.array_equal(sig, ref, equal_nan=True)
    assert np.array_equal(reg, reg_ref)


def test_counts_of_hand_checked_quotes():
    # an invalid quote stops at the finiteness tests: no arithmetic at all; a
    # price below intrinsic runs the status rule and nothing else
    w = dict(model=0, P=np.array([np.nan, 5.0]), S_or_F=np.array([100.0, 100.0]),
             K=np.array([90.0, 90.0]), T=np.array([1.0, 1.0]), r=np.array([0.0, 0.0]), q=None,
             flag=np.array([1, 1], np.int8))
    counts, reg, _ = count_ops.count(0, w)
    total = count_ops.flops(counts[:, -1])
    assert total[0] == 0 and list(reg) == [-1, -1]
    # status rule of an in-the-money call (log1p near the money, exp of r T,
    # sqrt, expm1 and exp of -|x|/2): no iteration was counted
    assert np.array_equal(counts[1, 0], counts[1, -1])
    f = dict(zip(count_ops.FIELDS, counts[1, -1]))
    assert (f["log1p"], f["exp"], f["expm1"], f["sqrt"], f["log"]) == (1, 2, 1, 1, 0)


def test_benchmark_figures_come_from_the_counted_build(grid_sample):
    import bench
    with open(os.path.join(ROOT, "oracle", "op_counts.json")) as f:
        stored = json.load(f)["workloads"][GRID]["method_flops_per_quote_by_path"]
    for path, v in stored.items():
        assert bench.ALG_FLOPS_PER_QUOTE[path] == pytest.approx(v, abs=0.05), path
    # and the stored figure is reproduced on another seeded sample (sampling
    # noise of a mean over thousands of quotes)
    s, _ = count_ops.summarise(grid_sample["model"], grid_sample)
    for path, v in s["method_flops_per_quote_by_path"].items():
        assert v == pytest.approx(stored[path], rel=0.03), path
