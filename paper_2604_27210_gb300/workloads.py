"""Seeded synthetic inputs for the five benchmark workloads.

This module only draws random numbers and lays them out; it holds none of the
pricing or inversion arithmetic.  Prices are filled in by a caller-supplied
price function (the oracle in the tests, the library's own pricing kernel in
the benchmark), so the same generator serves both sides.

All draws use numpy's PCG64 with the seed given, in the order documented in
each function.  Model codes: 0 Black-76, 1 Black-Scholes, 2 BSM.
"""
import numpy as np

BLACK76, BLACK_SCHOLES, BSM = 0, 1, 2


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _alternating_flags(n):
    f = np.ones(n, np.int8)
    f[1::2] = -1
    return f


def black76_quotes(n=4096, seed=0):
    """Black-76 quotes on a forward (4,096 quotes at the reference size).

    F = 100, K = F e^k with k ~ U[-1/2, 1/2], T ~ U[0.02, 2] years, r = 0.03,
    sigma_true ~ U[0.05, 1], calls at even and puts at odd indices.
    Draw order: k, T, sigma.
    """
    g = _rng(seed)
    k = g.uniform(-0.5, 0.5, n)
    T = g.uniform(0.02, 2.0, n)
    sigma = g.uniform(0.05, 1.0, n)
    F = np.full(n, 100.0)
    return dict(model=BLACK76, S_or_F=F, K=F * np.exp(k), T=T, r=np.full(n, 0.03), q=None,
                flag=_alternating_flags(n), sigma_true=sigma)


def bsm_grid(n_strikes=4096, n_maturities=4096, seed=1, below_fraction=0.05):
    """BSM quotes on a strike x maturity grid (4,096 x 4,096 at the reference size).

    Quote i = m * n_strikes + j (maturity-major, strikes contiguous).  S = 100,
    log-moneyness k_j = -3 + 6 j / (n_strikes - 1), K_j = S e^{k_j}, T_m
    log-spaced on [1/365, 5] years, r_i ~ U[0, 0.06], q_i ~ U[0, 0.05],
    sigma_i ~ U[0.01, 3].  Each quote is out of the money on its forward
    (call iff k_j >= (r_i - q_i) T_m).  A Bernoulli(below_fraction) mask flips
    a quote to the in-the-money side and prices it below its discounted
    intrinsic value by the factor 1 - (1e-6 + 1e-3 u), u ~ U[0, 1].
    Draw order: r, q, sigma, mask uniforms, u.
    """
    n = n_strikes * n_maturities
    g = _rng(seed)
    kj = -3.0 + 6.0 * np.arange(n_strikes) / max(n_strikes - 1, 1)
    Tm = np.exp(np.linspace(np.log(1.0 / 365.0), np.log(5.0), n_maturities))
    k = np.tile(kj, n_maturities)
    T = np.repeat(Tm, n_strikes)
    r = g.uniform(0.0, 0.06, n)
    q = g.uniform(0.0, 0.05, n)
    sigma = g.uniform(0.01, 3.0, n)
    mask = g.uniform(0.0, 1.0, n) < below_fraction
    u = g.uniform(0.0, 1.0, n)
    flag = np.where(k >= (r - q) * T, 1, -1).astype(np.int8)
    flag[mask] = -flag[mask]
    S = np.full(n, 100.0)
    return dict(model=BSM, S_or_F=S, K=S * np.exp(k), T=T, r=r, q=q, flag=flag,
                sigma_true=sigma, below_mask=mask, below_factor=1.0 - (1e-6 + 1e-3 * u))


def black76_fp32(n=67108864, seed=2):
    """Black-76 quotes with the distributions of black76_quotes, inputs in FP32.

    F, K, T, r are rounded to float32; the price (filled by fill_prices with
    the FP32 inputs widened to FP64) is rounded to float32 by the caller of
    fill_prices(..., price_dtype=np.float32).  Draw order: k, T, sigma.
    """
    w = black76_quotes(n, seed)
    for key in ("S_or_F", "K", "T", "r"):
        w[key] = w[key].astype(np.float32)
    return w


def chains(n_chains=10000, seed=3, min_len=8, max_len=65536):
    """Option chains of uneven length (10,000 chains at the reference size).

    len_c = floor(exp(U[ln min_len, ln max_len])); per chain F_c ~ U[10, 500],
    T_c ~ U[1/365, 3] years, r = 0.03; per quote k ~ U[-1/2, 1/2],
    K = F_c e^k, sigma ~ U[0.05, 1], calls at even and puts at odd positions.
    Returns flat arrays with chain offsets.  Draw order: lengths, F_c, T_c,
    then k and sigma for all quotes.
    """
    g = _rng(seed)
    lens = np.floor(np.exp(g.uniform(np.log(min_len), np.log(max_len), n_chains))).astype(np.int64)
    Fc = g.uniform(10.0, 500.0, n_chains)
    Tc = g.uniform(1.0 / 365.0, 3.0, n_chains)
    offsets = np.zeros(n_chains + 1, np.int64)
    np.cumsum(lens, out=offsets[1:])
    n = int(offsets[-1])
    k = g.uniform(-0.5, 0.5, n)
    sigma = g.uniform(0.05, 1.0, n)
    chain_of = np.repeat(np.arange(n_chains), lens)
    pos = np.arange(n) - offsets[chain_of]
    flag = np.where(pos % 2 == 0, 1, -1).astype(np.int8)
    F = Fc[chain_of]
    return dict(model=BLACK76, lens=lens, offsets=offsets, F_chain=Fc, T_chain=Tc,
                r_chain=np.full(n_chains, 0.03), S_or_F=F, K=F * np.exp(k), T=Tc[chain_of],
                r=np.full(n, 0.03), q=None, flag=flag, sigma_true=sigma)


def bsm_quotes(n=8388608, seed=4):
    """BSM quotes for differentiation (8,388,608 at the reference size).

    S = 100, K = S e^k with k ~ U[-1/2, 1/2], T ~ U[0.02, 2], r = 0.03,
    q ~ U[0, 0.05], sigma_true ~ U[0.05, 1], alternating call/put, and an
    upstream gradient grad_sigma ~ N(0, 1).  Draw order: k, T, q, sigma,
    grad_sigma.
    """
    g = _rng(seed)
    k = g.uniform(-0.5, 0.5, n)
    T = g.uniform(0.02, 2.0, n)
    q = g.uniform(0.0, 0.05, n)
    sigma = g.uniform(0.05, 1.0, n)
    gs = g.standard_normal(n)
    S = np.full(n, 100.0)
    return dict(model=BSM, S_or_F=S, K=S * np.exp(k), T=T, r=np.full(n, 0.03), q=q,
                flag=_alternating_flags(n), sigma_true=sigma, grad_sigma=gs)


def fill_prices(w, price_fn, price_dtype=np.float64):
    """Set w["P"] = price_fn(model, S_or_F, K, T, r, q, sigma, flag).

    Quotes under w["below_mask"] are priced at sigma = 0 (the discounted
    intrinsic value) and scaled by w["below_factor"].  Inputs are widened to
    FP64 before pricing; the result is cast to price_dtype.
    """
    f64 = lambda a: None if a is None else np.asarray(a, dtype=np.float64)
    sigma = w["sigma_true"]
    mask = w.get("below_mask")
    if mask is not None:
        sigma = np.where(mask, 0.0, sigma)
    P = np.asarray(price_fn(w["model"], f64(w["S_or_F"]), f64(w["K"]), f64(w["T"]), f64(w["r"]),
                            f64(w["q"]), sigma, w["flag"]), dtype=np.float64)
    if mask is not None:
        P = np.where(mask, P * w["below_factor"], P)
    w["P"] = P.astype(price_dtype)
    return w
