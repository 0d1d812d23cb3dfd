"""The seeded input generators (paper_2604_27210_gb300/workloads.py) follow the
recipes the benchmark and the parity tests are stated on: shapes, layouts,
ranges, flag patterns, the below-intrinsic perturbation, and determinism in
the seed.  CPU only."""
import numpy as np

from oracle import oracle as orc
from paper_2604_27210_gb300 import workloads as wl


def test_bsm_grid_layout_and_ranges():
    ns, nm = 64, 32
    w = wl.bsm_grid(ns, nm, seed=1)
    n = ns * nm
    assert w["model"] == wl.BSM and all(w[k].size == n for k in ("S_or_F", "K", "T", "r", "q", "flag"))
    assert np.all(w["S_or_F"] == 100.0)
    # maturity-major: strikes contiguous and shared by every maturity row
    k = np.log(w["K"] / 100.0).reshape(nm, ns)
    assert np.allclose(k, k[0]) and np.isclose(k[0, 0], -3.0) and np.isclose(k[0, -1], 3.0)
    assert np.all(np.diff(k[0]) > 0)
    T = w["T"].reshape(nm, ns)
    assert np.all(T == T[:, :1]) and np.isclose(T[0, 0], 1 / 365) and np.isclose(T[-1, 0], 5.0)
    assert np.allclose(np.diff(np.log(T[:, 0])), np.log(5 * 365) / (nm - 1))  # log-spaced
    assert w["r"].min() >= 0 and w["r"].max() < 0.06 and w["q"].min() >= 0 and w["q"].max() < 0.05
    assert w["sigma_true"].min() >= 0.01 and w["sigma_true"].max() < 3.0
    # out of the money on the forward, except the masked quotes (flipped in the money)
    otm = np.where(np.log(w["K"] / 100.0) >= (w["r"] - w["q"]) * w["T"], 1, -1)
    m = w["below_mask"]
    assert np.array_equal(w["flag"][~m], otm[~m]) and np.array_equal(w["flag"][m], -otm[m])
    f = w["below_factor"]
    assert np.all((f <= 1 - 1e-6) & (f > 1 - 1e-6 - 1e-3))


def test_bsm_grid_mask_fraction_and_pricing():
    w = wl.fill_prices(wl.bsm_grid(4096, 16, seed=2), orc.price_f64)
    m = w["below_mask"]
    assert abs(m.mean() - 0.05) < 0.005
    # masked quotes: the discounted intrinsic value (price at sigma = 0) times the factor
    intr = orc.price_f64(wl.BSM, w["S_or_F"][m], w["K"][m], w["T"][m], w["r"][m], w["q"][m],
                         np.zeros(m.sum()), w["flag"][m])
    assert np.allclose(w["P"][m], intr * w["below_factor"][m], rtol=1e-15, atol=0)
    assert np.all(w["P"][m] < intr)
    st = orc.status(wl.BSM, w["P"], w["S_or_F"], w["K"], w["T"], w["r"], w["q"], w["flag"])[0]
    assert np.all(st[m][intr > 1e-300] == orc.BELOW_INTRINSIC)


def test_black76_quotes_and_fp32_inputs():
    w = wl.black76_quotes(4096, seed=0)
    assert w["model"] == wl.BLACK76 and w["q"] is None
    assert np.all(w["S_or_F"] == 100.0) and np.all(w["r"] == 0.03)
    k = np.log(w["K"] / 100.0)
    assert k.min() >= -0.5 and k.max() < 0.5
    assert w["T"].min() >= 0.02 and w["T"].max() < 2.0
    assert w["sigma_true"].min() >= 0.05 and w["sigma_true"].max() < 1.0
    assert np.all(w["flag"][0::2] == 1) and np.all(w["flag"][1::2] == -1)
    w32 = wl.black76_fp32(4096, seed=0)
    assert all(w32[k].dtype == np.float32 for k in ("S_or_F", "K", "T", "r"))
    assert np.array_equal(w32["K"], w["K"].astype(np.float32))  # the same draws, rounded


def test_chains_lengths_offsets_and_per_chain_values():
    c = wl.chains(200, seed=3, max_len=5000)
    lens, off = c["lens"], c["offsets"]
    assert lens.min() >= 8 and lens.max() < 5000 and off[0] == 0 and np.array_equal(np.diff(off), lens)
    n = int(off[-1])
    assert c["K"].size == n and c["S_or_F"].size == n
    chain_of = np.repeat(np.arange(200), lens)
    assert np.array_equal(c["S_or_F"], c["F_chain"][chain_of]) and np.array_equal(c["T"], c["T_chain"][chain_of])
    assert c["F_chain"].min() >= 10 and c["F_chain"].max() < 500
    assert c["T_chain"].min() >= 1 / 365 and c["T_chain"].max() < 3
    pos = np.arange(n) - off[chain_of]
    assert np.array_equal(c["flag"], np.where(pos % 2 == 0, 1, -1))
    # log-uniform lengths: the log of the lengths spreads over [ln 8, ln 5000)
    ll = np.log(lens)
    assert ll.min() < np.log(8) + 1 and ll.max() > np.log(5000) - 1


def test_bsm_quotes_for_differentiation():
    w = wl.bsm_quotes(4096, seed=4)
    assert w["model"] == wl.BSM and np.all(w["r"] == 0.03)
    assert w["q"].min() >= 0 and w["q"].max() < 0.05
    assert w["grad_sigma"].size == 4096 and abs(w["grad_sigma"].mean()) < 0.1
    assert np.all(w["flag"][0::2] == 1) and np.all(w["flag"][1::2] == -1)


def test_generators_are_deterministic_in_the_seed():
    for gen in (lambda s: wl.bsm_grid(32, 8, seed=s), lambda s: wl.black76_quotes(256, seed=s),
                lambda s: wl.chains(10, seed=s, max_len=100), lambda s: wl.bsm_quotes(256, seed=s)):
        a, b, c = gen(7), gen(7), gen(8)
        assert np.array_equal(a["K"], b["K"]) and np.array_equal(a["sigma_true"], b["sigma_true"])
        m = min(a["sigma_true"].size, c["sigma_true"].size)
        assert not np.array_equal(a["sigma_true"][:m], c["sigma_true"][:m])
