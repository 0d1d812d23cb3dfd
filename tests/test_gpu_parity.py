"""Parity of the CUDA library against the oracle (needs a GPU).

Floating-point tolerances (the target accuracy, read with the conditioning
of each quote):
  - sigma, FP64 paths (LBR, Halley, mixed): relative error <= 1e-12 wherever
    the normalised vega b' > 1e-8; elsewhere (solved quotes) the error is
    bounded by 1e-12 + 16 eps (1 + kappa), kappa = beta / (s b').
  - sigma, pure FP32 paths: relative error <= 1e-5 (FP32 LBR) or 1e-4 (the
    plain-Phi FP32 Halley) where b' > 1e-8 and kappa <= 1e3 (their FP32 solve
    keeps the FP64 reduced price's rounding, amplified by kappa).
  - price round trip: relative <= 1e-13 where b' > 1e-8.
  - status: bit-identical for every quote.
"""
import ctypes

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2604_27210_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -52


@pytest.fixture(scope="module")
def fv():
    from paper_2604_27210_gb300 import fv as mod
    return mod


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    return torch, torch.device("cuda:0")


def _dev(torch_dev, a):
    torch, dev = torch_dev
    return torch.tensor(np.ascontiguousarray(a), device=dev)


def _np(t):
    return t.cpu().numpy()


class _Conditioning(np.ndarray):
    """kappa per quote, carrying `amb`: the quotes whose status quantities lie
    within 16 ulp of a threshold of the FP64 status rule."""


def _iv_ref(w, model=None):
    model = w["model"] if model is None else model
    f = lambda k: None if w.get(k) is None else np.asarray(w[k], dtype=np.float64)
    sig, st = orc.iv(model, f("P"), f("S_or_F"), f("K"), f("T"), f("r"), f("q"), w["flag"])
    v, kap = orc.conditioning(model, f("P"), f("S_or_F"), f("K"), f("T"), f("r"), f("q"),
                              w["flag"], sig)
    margin = orc.status(model, f("P"), f("S_or_F"), f("K"), f("T"), f("r"), f("q"), w["flag"])[3]
    kap = kap.view(_Conditioning)
    kap.amb = margin <= 16.0
    return sig, st, v, kap


def _check_sigma(got, ref, st, v, kap, tol_gate=1e-12, tol_rest=None, name=""):
    # A quote whose price exceeds its intrinsic value by 64 ulp of it (the
    # status rule's at-intrinsic threshold) to within a few ulp may take
    # sigma = 0 on one side and a positive sigma on the other: the kernels' and
    # the oracle's libm differ in the last place.  Those quotes (and any other
    # within 16 ulp of a threshold) need only a finite sigma >= 0.
    amb = getattr(kap, "amb", np.zeros(got.shape, bool))
    assert amb.mean() <= 1e-3, "%s: %d ambiguous quotes" % (name, amb.sum())
    okq = st == orc.OK
    assert np.all(np.isfinite(got[okq & amb]) & (got[okq & amb] >= 0)), name
    st = np.where(amb & okq, 255, st)  # leave them out below
    solved = (st == orc.OK) & (ref > 0)
    # quotes at intrinsic and failures: exact values
    assert np.all(got[(st == orc.OK) & (ref == 0)] == 0.0), name
    assert np.all(np.isnan(got[(st != orc.OK) & (st != 255)])), name
    assert np.all(np.isfinite(got[solved]) & (got[solved] > 0)), name
    rel = np.abs(got[solved] - ref[solved]) / ref[solved]
    # FP64 paths: every quote with b' > 1e-8 (their ill-conditioned quotes'
    # reduced price is refined in double-double); FP32 paths: kappa <= 1e3 too
    gate = v[solved] > 1e-8
    if tol_gate > 1e-12:
        gate &= kap[solved] <= 1e3
    if gate.any():
        assert rel[gate].max() <= tol_gate, "%s: gated max rel %.3g" % (name, rel[gate].max())
    if tol_rest is not None:
        k = np.nan_to_num(kap[solved], nan=np.inf, posinf=np.inf)
        bound = tol_rest + 16 * EPS * (1 + k)
        bad = rel > bound
        assert not bad.any(), "%s: %d quotes beyond the conditioning bound (worst %.3g)" % (
            name, bad.sum(), rel[bad].max())
    return rel, gate


def _args(torch_dev, w, keys=("P", "S_or_F", "K", "T", "r", "q")):
    return [None if w.get(k) is None else _dev(torch_dev, w[k]) for k in keys]


# ---------------------------------------------------------------------------
# normalised Black function
# ---------------------------------------------------------------------------
def test_erfcx_against_binary128(fv, torch_dev):
    # the kernels' own erfcx: table below z = 128, asymptotic series above,
    # reflection below zero; every piece edge and its neighbours included
    torch, dev = torch_dev
    g = np.random.default_rng(9)
    edges = np.array([k / 16 for k in range(9)] + [2.0 ** e * (1 + j / 16) for e in range(-1, 7)
                                                   for j in range(16)] + [128.0])
    pos = np.concatenate([g.uniform(0, 0.5, 20000), np.exp(g.uniform(np.log(0.5), np.log(128), 50000)),
                          np.exp(g.uniform(np.log(128), np.log(1e300), 20000)), edges,
                          np.nextafter(edges, 0), np.nextafter(edges, np.inf), [0.0, 5e-324]])
    neg = -np.concatenate([g.uniform(0, 26.6, 40000), np.exp(g.uniform(np.log(1e-300), np.log(1), 5000))])
    z = np.concatenate([pos, neg])
    got = _np(fv.fv_math(fv.FV_MATH_ERFCX, torch.tensor(z, device=dev)))
    ref = orc.erfcx(z)
    fin = np.isfinite(ref)
    rel = np.abs(got[fin] - ref[fin]) / ref[fin]
    zf = z[fin]
    assert rel[zf >= 0].max() <= 4e-16, rel[zf >= 0].max()
    assert rel[zf < 0].max() <= 8e-16, rel[zf < 0].max()
    assert np.array_equal(np.isinf(got), np.isinf(ref))
    sp = _np(fv.fv_math(fv.FV_MATH_ERFCX, torch.tensor([np.inf, -np.inf, -27.0, np.nan, -0.0],
                                                        dtype=torch.float64, device=dev)))
    assert sp[0] == 0 and sp[1] == np.inf and sp[2] == np.inf and np.isnan(sp[3]) and sp[4] == 1.0


def test_erfcx_of_w_over_sqrt2_against_binary128(fv, torch_dev):
    # the solvers' form erfcx(w/sqrt2): its piece index comes from an FP32 view
    # of w/sqrt2, so arguments next to every piece edge are included.  The
    # reference is the oracle's erfcx at z = fl(w/sqrt2) moved to the exact
    # w/sqrt2 by the derivative erfcx'(z) = 2 z erfcx(z) - 2/sqrt(pi).
    torch, dev = torch_dev
    g = np.random.default_rng(13)
    edges = np.array([k / 16 for k in range(1, 9)] + [2.0 ** e * (1 + j / 16) for e in range(-1, 7)
                                                      for j in range(16)] + [128.0])
    we = edges * np.sqrt(2.0)
    w = np.concatenate([g.uniform(0, 0.8, 20000), np.exp(g.uniform(np.log(0.7), np.log(181), 50000)),
                        np.exp(g.uniform(np.log(181), np.log(1e300), 5000)), we, np.nextafter(we, 0),
                        np.nextafter(we, np.inf), we * (1 - 3e-7), we * (1 + 3e-7), [0.0, 5e-324],
                        -g.uniform(0, 37.6, 20000)])
    got = _np(fv.fv_math(fv.FV_MATH_ERFCX_SQRT2, torch.tensor(w, device=dev)))
    k = np.longdouble(1) / np.sqrt(np.longdouble(2))
    z_ld = w.astype(np.longdouble) * k
    z = z_ld.astype(np.float64)
    delta = (z_ld - z.astype(np.longdouble)).astype(np.float64)
    fz = orc.erfcx(z)
    # (beyond z = 10 the derivative's two terms cancel: take erfcx'/erfcx ~ -1/z)
    big = z > 10
    with np.errstate(over="ignore", invalid="ignore"):
        ref = np.where(big, fz * (1 - delta / np.where(big, z, 1.0)),
                       fz + delta * (2 * z * fz - 2 / np.sqrt(np.pi)))
    fin = np.isfinite(ref) & (ref > 0)
    rel = np.abs(got[fin] - ref[fin]) / ref[fin]
    wf = w[fin]
    # the table's 1.2 ulp, the rounded constant 1/sqrt2 inside v = w/sqrt2 - c
    # (z |d ln erfcx/dz| <= ~1 of its 0.35 ulp) and v's rounding, and the
    # reference's own final rounding
    assert rel[wf >= 0].max() <= 6e-16, rel[wf >= 0].max()
    assert rel[wf < 0].max() <= 1e-15, rel[wf < 0].max()


def test_log_against_extended_precision(fv, torch_dev):
    # the kernels' own FP64 log (Tang's table-driven method) against numpy's
    # long double log (binary128 on Arm, 64-bit mantissa on x86)
    torch, dev = torch_dev
    g = np.random.default_rng(10)
    y = np.concatenate([np.exp(g.uniform(-708, 709, 100000)), 1 + g.uniform(-0.02, 0.02, 20000),
                        1 + np.exp(g.uniform(-36, -5, 5000)), 1 - np.exp(g.uniform(-36, -5, 5000)),
                        [2.2250738585072014e-308, 1.7976931348623157e308, 0.5, 2.0, 1.0]])
    got = _np(fv.fv_math(fv.FV_MATH_LOG, torch.tensor(y, device=dev)))
    ref = np.log(y.astype(np.longdouble))
    nz = ref != 0
    rel = np.abs((got[nz] - ref[nz]) / ref[nz]).astype(np.float64)
    # final rounding (1/2 ulp) plus the second sum's rounding relative to a
    # result that can be as small as ln(1 + 1/256) (up to ~1/2 ulp more)
    assert rel.max() <= 1.5 * 2.0 ** -52, rel.max()
    assert np.all(got[~nz] == 0)
    sp = _np(fv.fv_math(fv.FV_MATH_LOG, torch.tensor([0.0, -1.0, np.inf, np.nan, 5e-324],
                                                      dtype=torch.float64, device=dev)))
    assert sp[0] == -np.inf and np.isnan(sp[1]) and sp[2] == np.inf and np.isnan(sp[3])
    assert sp[4] == pytest.approx(np.log(5e-324), rel=1e-15)


def test_exp_against_extended_precision(fv, torch_dev):
    # the kernels' own FP64 exp (Tang's table-driven method) against numpy's
    # long double exp; subnormal, overflowing and NaN arguments included
    torch, dev = torch_dev
    g = np.random.default_rng(11)
    v = np.concatenate([g.uniform(-708, 709.5, 100000), g.uniform(-1e-3, 1e-3, 20000),
                        g.uniform(-30, 5, 20000), [0.0, -0.0, 1.0, -1.0, 709.7, -708.3]])
    got = _np(fv.fv_math(fv.FV_MATH_EXP, torch.tensor(v, device=dev)))
    ref = np.exp(v.astype(np.longdouble))
    rel = np.abs((got - ref) / ref).astype(np.float64)
    # Tang's bound: the final rounding plus the polynomial's, about 0.54 ulp
    assert rel.max() <= 2.0 ** -52, rel.max()
    sp = _np(fv.fv_math(fv.FV_MATH_EXP, torch.tensor([-745.3, -740.0, 710.0, np.inf, -np.inf, np.nan],
                                                      dtype=torch.float64, device=dev)))
    assert sp[0] == 0 and sp[1] == pytest.approx(np.exp(-740.0), rel=1e-12) and sp[2] == np.inf
    assert sp[3] == np.inf and sp[4] == 0 and np.isnan(sp[5])


def test_expm1_and_log1p_against_extended_precision(fv, torch_dev):
    # expm1 from the exponential's reduction, log1p as the logarithm of the
    # exact sum 1 + z: the status rule's intrinsic value and x near the money
    torch, dev = torch_dev
    g = np.random.default_rng(12)
    v = np.concatenate([-np.exp(g.uniform(np.log(1e-300), np.log(708), 50000)),
                        g.uniform(-0.01, 0.01, 20000), g.uniform(-1.5, 1.5, 20000),
                        g.uniform(0, 709.6, 10000), [0.0, -0.0, -708.29, 709.69]])
    got = _np(fv.fv_math(fv.FV_MATH_EXPM1, torch.tensor(v, device=dev)))
    ref = np.expm1(v.astype(np.longdouble))
    nz = ref != 0
    rel = np.abs((got[nz] - ref[nz]) / ref[nz]).astype(np.float64)
    assert rel.max() <= 1.25 * 2.0 ** -52, rel.max()
    assert np.all(got[~nz] == 0)
    sp = _np(fv.fv_math(fv.FV_MATH_EXPM1, torch.tensor([-708.4, -1e300, 710.0, np.inf, -np.inf, np.nan],
                                                        dtype=torch.float64, device=dev)))
    assert sp[0] == -1 and sp[1] == -1 and sp[2] == np.inf and sp[3] == np.inf and sp[4] == -1
    assert np.isnan(sp[5])
    u = np.concatenate([g.uniform(-0.5, 1.0, 50000), np.exp(g.uniform(np.log(1e-300), 0, 20000)),
                        -np.exp(g.uniform(np.log(1e-300), np.log(0.9999), 20000)),
                        np.exp(g.uniform(0, 700, 10000)), [0.0, -0.5, 1.0, 1.0 / 512, -1.0 / 512]])
    got = _np(fv.fv_math(fv.FV_MATH_LOG1P, torch.tensor(u, device=dev)))
    ref = np.log1p(u.astype(np.longdouble))
    nz = ref != 0
    rel = np.abs((got[nz] - ref[nz]) / ref[nz]).astype(np.float64)
    assert rel.max() <= 1.5 * 2.0 ** -52, rel.max()
    assert np.all(got[~nz] == 0)
    sp = _np(fv.fv_math(fv.FV_MATH_LOG1P, torch.tensor([-1.0, -2.0, np.inf, np.nan, 5e-324],
                                                        dtype=torch.float64, device=dev)))
    assert sp[0] == -np.inf and np.isnan(sp[1]) and sp[2] == np.inf and np.isnan(sp[3])
    assert sp[4] == 5e-324


def test_normalised_black_against_binary128(fv, torch_dev):
    xs = np.concatenate([-np.logspace(-8, np.log10(40), 60), [0.0], np.logspace(-8, np.log10(40), 60)])
    ss = np.logspace(-4, np.log10(50), 90)
    X, S = np.meshgrid(xs, ss, indexing="ij")
    X, S = X.ravel(), S.ravel()
    for th in (1, -1):
        thv = np.full(X.size, th, np.int8)
        ref = orc.normalised_black(X, S, thv)
        got = _np(fv.fv_normalised_black(_dev(torch_dev, X), _dev(torch_dev, S), _dev(torch_dev, thv)))
        m = ref > 1e-300
        rel = np.abs(got[m] - ref[m]) / ref[m]
        # the erfcx difference loses log10(|h|/2t) digits in the deep wing
        assert rel.max() <= 2e-12
        # where b' is not negligible (|h| < 6) and s <= 10 (beyond it the
        # exponent -(h^2+t^2)/2 alone carries |.| eps of relative error)
        h = np.abs(X[m]) / S[m]
        core = (h < 6) & (S[m] <= 10)
        assert rel[core].max() <= 1e-13
    # s = 0 is the intrinsic value; s = inf the upper bound
    x = np.array([0.3, -0.3, 0.0])
    z = _np(fv.fv_normalised_black(_dev(torch_dev, x), _dev(torch_dev, np.zeros(3)),
                                   _dev(torch_dev, np.ones(3, np.int8))))
    np.testing.assert_allclose(z, np.maximum(2 * np.sinh(x / 2), 0), rtol=4 * EPS, atol=0)


# ---------------------------------------------------------------------------
# implied volatility: Black-76 quotes (4,096 at the reference size)
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def black76():
    w = wl.fill_prices(wl.black76_quotes(4096, seed=0), orc.price)
    return w, _iv_ref(w)


@pytest.mark.parametrize("solver", ["lbr", "halley"])
def test_iv_black76_fp64(fv, torch_dev, black76, solver):
    w, (ref, st_ref, v, kap) = black76
    P, F, K, T, r, _ = _args(torch_dev, w)
    s, st = fv.fv_implied_vol(fv.FV_BLACK76, fv.FV_LBR if solver == "lbr" else fv.FV_HALLEY, P, F,
                              K, T, r, None, _dev(torch_dev, w["flag"]))
    assert np.array_equal(_np(st), st_ref)
    _check_sigma(_np(s), ref, st_ref, v, kap, tol_rest=1e-12, name=solver)


def test_iv_round_trip_price(fv, torch_dev, black76):
    w, (ref, st_ref, v, kap) = black76
    P, F, K, T, r, _ = _args(torch_dev, w)
    flag = _dev(torch_dev, w["flag"])
    s, st = fv.fv_implied_vol(fv.FV_BLACK76, fv.FV_LBR, P, F, K, T, r, None, flag)
    back = _np(fv.fv_price(fv.FV_BLACK76, flag, F, K, T, r, None, s))
    m = (st_ref == orc.OK) & (v > 1e-8) & (ref > 0)
    rel = np.abs(back[m] - w["P"][m]) / w["P"][m]
    assert rel.max() <= 1e-13


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
def test_iv_black76_reduced_precision(fv, torch_dev, black76, prec):
    w, (ref, st_ref, v, kap) = black76
    P, F, K, T, r, _ = _args(torch_dev, w)
    p = fv.FV_MIXED if prec == "mixed" else fv.FV_FP32
    s, st = fv.fv_implied_vol_ex(fv.FV_BLACK76, fv.FV_LBR, p, P, F, K, T, r, None,
                                 _dev(torch_dev, w["flag"]))
    assert np.array_equal(_np(st), st_ref)
    if prec == "mixed":
        _check_sigma(_np(s), ref, st_ref, v, kap, tol_gate=1e-12, tol_rest=1e-12, name=prec)
    else:
        _check_sigma(_np(s), ref, st_ref, v, kap, tol_gate=1e-5, name=prec)


# ---------------------------------------------------------------------------
# BSM strike x maturity grid, 5% below intrinsic (reduced grid; full size below)
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def bsm_grid_small():
    w = wl.fill_prices(wl.bsm_grid(512, 96, seed=1), orc.price)
    return w, _iv_ref(w)


@pytest.mark.parametrize("mode", ["lbr", "halley", "mixed", "fp32", "halley32"])
def test_iv_bsm_grid(fv, torch_dev, bsm_grid_small, mode):
    w, (ref, st_ref, v, kap) = bsm_grid_small
    assert (st_ref == orc.BELOW_INTRINSIC).sum() > 0.03 * st_ref.size
    args = _args(torch_dev, w)
    flag = _dev(torch_dev, w["flag"])
    if mode in ("lbr", "halley"):
        s, st = fv.fv_implied_vol(fv.FV_BSM, fv.FV_LBR if mode == "lbr" else fv.FV_HALLEY, *args, flag)
    elif mode == "halley32":
        s, st = fv.fv_implied_vol_ex(fv.FV_BSM, fv.FV_HALLEY, fv.FV_FP32, *args, flag)
    else:
        s, st = fv.fv_implied_vol_ex(fv.FV_BSM, fv.FV_LBR,
                                     fv.FV_MIXED if mode == "mixed" else fv.FV_FP32, *args, flag)
    assert np.array_equal(_np(st), st_ref)
    if mode == "fp32":
        _check_sigma(_np(s), ref, st_ref, v, kap, tol_gate=1e-5, name=mode)
    elif mode == "halley32":
        # the paper's float32 throughput path (plain-Phi residual): looser
        _check_sigma(_np(s), ref, st_ref, v, kap, tol_gate=1e-4, name=mode)
    else:
        _check_sigma(_np(s), ref, st_ref, v, kap, tol_rest=1e-12, name=mode)


def test_halley32_black76(fv, torch_dev, black76):
    w, (ref, st_ref, v, kap) = black76
    P, F, K, T, r, _ = _args(torch_dev, w)
    s, st = fv.fv_implied_vol_ex(fv.FV_BLACK76, fv.FV_HALLEY, fv.FV_FP32, P, F, K, T, r, None,
                                 _dev(torch_dev, w["flag"]))
    assert np.array_equal(_np(st), st_ref)
    # the paper's float32 throughput path: the plain-Phi residual loses about a
    # digit to cancellation, so its bar is 1e-4 (the LBR FP32 path meets 1e-5)
    _check_sigma(_np(s), ref, st_ref, v, kap, tol_gate=1e-4, name="halley32")


def test_strided_broadcast_matches_arrays(fv, torch_dev):
    torch, dev = torch_dev
    # the paper's quick-use call shape: scalar S, t, r; arrays of strikes and flags
    w = wl.fill_prices(wl.bsm_quotes(3000, seed=31), orc.price)
    n = w["K"].size
    scal = dict(S_or_F=100.0, T=0.25, r=0.05, q=0.01)
    full = {k: np.full(n, v) for k, v in scal.items()}
    full.update(K=w["K"], flag=w["flag"], model=2)
    full["P"] = orc.price(2, full["S_or_F"], full["K"], full["T"], full["r"], full["q"],
                          w["sigma_true"], full["flag"])
    ref, st_ref, v, kap = _iv_ref(full)
    one = lambda x: torch.tensor([x], dtype=torch.float64, device=dev)
    for prec in (fv.FV_FP64, fv.FV_MIXED):
        s_b, st_b = fv.fv_implied_vol_strided(2, fv.FV_LBR, prec, _dev(torch_dev, full["P"]),
                                              one(100.0), _dev(torch_dev, full["K"]), one(0.25),
                                              one(0.05), one(0.01), _dev(torch_dev, full["flag"]))
        s_a, st_a = fv.fv_implied_vol_ex(2, fv.FV_LBR, prec, *_args(torch_dev, full),
                                         _dev(torch_dev, full["flag"]))
        assert torch.equal(st_a, st_b) and np.array_equal(_np(st_b), st_ref)
        assert torch.equal(s_a.nan_to_num(-1), s_b.nan_to_num(-1))
        _check_sigma(_np(s_b), ref, st_ref, v, kap, tol_rest=1e-12)
    # a negative stride is an argument error
    lib = fv.library()
    import ctypes
    st = (ctypes.c_int64 * 7)(1, 1, 1, 1, 1, -1, 1)
    p = ctypes.c_void_p(s_b.data_ptr())
    assert lib.fv_implied_vol_strided(2, 0, 0, 0, p, p, p, p, p, p, p, st, n, p, p, None) == fv.FV_ERR_ARG


@pytest.mark.parametrize("n", [8192, 100000])
def test_iv_fp32_inputs(fv, torch_dev, n):
    # FP32 inputs; the oracle inverts the same values widened to FP64 (100,000
    # quotes: the medium-batch tiles of every precision)
    w = wl.black76_fp32(n, seed=2)
    wl.fill_prices(w, orc.price, price_dtype=np.float32)
    ref, st_ref, v, kap = _iv_ref(w)
    torch, dev = torch_dev
    args = [torch.tensor(w[k], device=dev) for k in ("P", "S_or_F", "K", "T", "r")]
    flag = _dev(torch_dev, w["flag"])
    for prec, tol in ((fv.FV_FP64, 1e-12), (fv.FV_MIXED, 1e-12), (fv.FV_FP32, 1e-5)):
        s, st = fv.fv_implied_vol_ex(fv.FV_BLACK76, fv.FV_LBR, prec, *args, None, flag)
        assert np.array_equal(_np(st), st_ref)
        _check_sigma(_np(s), ref, st_ref, v, kap, tol_gate=tol, name=str(prec))


# ---------------------------------------------------------------------------
# price, Greeks, adjoint
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("model", [0, 1, 2])
def test_price_against_oracle(fv, torch_dev, model):
    w = wl.bsm_quotes(8192, seed=5)
    q = w["q"] if model == 2 else None
    ref = orc.price(model, w["S_or_F"], w["K"], w["T"], w["r"], q, w["sigma_true"], w["flag"])
    got = _np(fv.fv_price(model, _dev(torch_dev, w["flag"]), _dev(torch_dev, w["S_or_F"]),
                          _dev(torch_dev, w["K"]), _dev(torch_dev, w["T"]), _dev(torch_dev, w["r"]),
                          None if q is None else _dev(torch_dev, q), _dev(torch_dev, w["sigma_true"])))
    m = ref > 1e-300
    assert (np.abs(got[m] - ref[m]) / ref[m]).max() <= 1e-12


def test_price_grid_wings(fv, torch_dev, bsm_grid_small):
    w, (ref, st_ref, v, kap) = bsm_grid_small
    sig = np.where(w["below_mask"], 0.0, w["sigma_true"])
    pref = orc.price(2, w["S_or_F"], w["K"], w["T"], w["r"], w["q"], sig, w["flag"])
    got = _np(fv.fv_price(2, _dev(torch_dev, w["flag"]), *[_dev(torch_dev, w[k]) for k in
                                                           ("S_or_F", "K", "T", "r", "q")],
                          _dev(torch_dev, sig)))
    m = pref > 1e-300
    assert (np.abs(got[m] - pref[m]) / pref[m]).max() <= 2e-12


@pytest.mark.parametrize("model", [0, 1, 2])
def test_greeks_against_oracle(fv, torch_dev, model):
    w = wl.bsm_quotes(4096, seed=6)
    q = w["q"] if model == 2 else None
    refs = orc.greeks(model, w["S_or_F"], w["K"], w["T"], w["r"], q, w["sigma_true"], w["flag"])
    got = fv.fv_greeks(model, _dev(torch_dev, w["flag"]), _dev(torch_dev, w["S_or_F"]),
                       _dev(torch_dev, w["K"]), _dev(torch_dev, w["T"]), _dev(torch_dev, w["r"]),
                       None if q is None else _dev(torch_dev, q), _dev(torch_dev, w["sigma_true"]))
    for name, ref in zip(("delta", "gamma", "vega", "theta", "rho"), refs):
        g = _np(got[name])
        scale = np.maximum(np.abs(ref), 1e-12)
        assert (np.abs(g - ref) / scale).max() <= 1e-12, name


@pytest.mark.parametrize("model", [0, 2])
def test_adjoint_against_oracle_and_fd(fv, torch_dev, model):
    w = wl.bsm_quotes(2048, seed=7)
    if model == 0:
        w["q"] = None
    w = wl.fill_prices(w, orc.price)
    ins = _args(torch_dev, w)
    flag = _dev(torch_dev, w["flag"])
    s, st = fv.fv_implied_vol(model, fv.FV_LBR, *ins, flag)
    gs = _dev(torch_dev, w["grad_sigma"])
    adj = fv.fv_iv_adjoint(model, *ins, flag, s, st, gs)
    s_np, st_np = _np(s), _np(st)
    refs = orc.iv_grad(model, w["S_or_F"], w["K"], w["T"], w["r"], w["q"], w["flag"], s_np, st_np,
                       w["grad_sigma"])
    v, kap = orc.conditioning(model, w["P"], w["S_or_F"], w["K"], w["T"], w["r"], w["q"], w["flag"],
                              s_np)
    ok = (st_np == orc.OK) & (s_np > 0) & (v > 1e-8)
    for name, ref in zip(("P", "S", "K", "T", "r", "q"), refs):
        g = _np(adj[name])
        scale = np.maximum(np.abs(ref[ok]), 1e-300)
        assert (np.abs(g[ok] - ref[ok]) / scale).max() <= 1e-11, name
    # central finite differences of the GPU implied volatility (h = 1e-6 relative)
    keys = ["P", "S_or_F", "K", "T", "r"] + (["q"] if model == 2 else [])
    names = ["P", "S", "K", "T", "r", "q"]
    for j, key in enumerate(keys):
        x0 = np.asarray(w[key], dtype=np.float64)
        h = 1e-6 * np.abs(x0) if key in ("P", "S_or_F", "K", "T") else np.full(x0.size, 1e-6)
        outs = []
        for sgn in (1, -1):
            ww = dict(w)
            ww[key] = x0 + sgn * h
            s_h, _ = fv.fv_implied_vol(model, fv.FV_LBR, *_args(torch_dev, ww), flag)
            outs.append(_np(s_h))
        fd = (outs[0] - outs[1]) / (2 * h) * w["grad_sigma"]
        g = _np(adj[names[j]])
        m = ok & (kap < 1e2)
        np.testing.assert_allclose(g[m], fd[m], rtol=2e-5, atol=1e-9, err_msg=key)


def test_autograd_function(fv, torch_dev):
    torch, dev = torch_dev
    w = wl.fill_prices(wl.bsm_quotes(1024, seed=8), orc.price)
    ins = [torch.tensor(w[k], device=dev, requires_grad=True) for k in
           ("P", "S_or_F", "K", "T", "r", "q")]
    flag = _dev(torch_dev, w["flag"])
    sigma = fv.implied_volatility_autograd(*ins, flag, model=fv.FV_BSM)
    g = torch.tensor(w["grad_sigma"], device=dev)
    (sigma * g).sum().backward()
    s2, st2 = fv.fv_implied_vol(fv.FV_BSM, fv.FV_LBR, *[t.detach() for t in ins], flag)
    assert torch.equal(sigma.detach().nan_to_num(-1), s2.nan_to_num(-1))
    adj = fv.fv_iv_adjoint(fv.FV_BSM, *[t.detach() for t in ins], flag, s2, st2, g)
    for t, name in zip(ins, ("P", "S", "K", "T", "r", "q")):
        assert torch.equal(t.grad, adj[name]), name


# ---------------------------------------------------------------------------
# batches of option chains
# ---------------------------------------------------------------------------
def _chain_tensors(torch_dev, c):
    torch, dev = torch_dev
    chains = []
    for j in range(len(c["lens"])):
        a, b = c["offsets"][j], c["offsets"][j + 1]
        chains.append(dict(price=_dev(torch_dev, c["P"][a:b]), K=_dev(torch_dev, c["K"][a:b]),
                           flag=_dev(torch_dev, c["flag"][a:b]),
                           sigma=torch.empty(b - a, dtype=torch.float64, device=dev),
                           status=torch.empty(b - a, dtype=torch.uint8, device=dev),
                           S_or_F=c["F_chain"][j], T=c["T_chain"][j], r=c["r_chain"][j]))
    return chains


@pytest.mark.parametrize("autotune", [False, True])
def test_chains_match_flat_and_oracle(fv, torch_dev, autotune):
    c = wl.fill_prices(wl.chains(120, seed=3, max_len=3000), orc.price)
    chains = _chain_tensors(torch_dev, c)
    plan = fv.fv_chains_plan_create(fv.FV_BLACK76, chains, autotune=autotune)
    for ch in chains:
        ch["sigma"].fill_(-7.0)
        ch["status"].fill_(9)
    plan.run()
    sig = np.concatenate([_np(ch["sigma"]) for ch in chains])
    st = np.concatenate([_np(ch["status"]) for ch in chains])
    # the flat kernel over the concatenated arrays: identical statuses, sigma
    # within rounding (two separately compiled kernels may contract FMAs
    # differently)
    s_flat, st_flat = fv.fv_implied_vol(fv.FV_BLACK76, fv.FV_LBR,
                                        *_args(torch_dev, c, ("P", "S_or_F", "K", "T", "r")), None,
                                        _dev(torch_dev, c["flag"]))
    assert np.array_equal(st, _np(st_flat))
    s_flat = _np(s_flat)
    assert np.array_equal(np.isnan(sig), np.isnan(s_flat))
    ok = ~np.isnan(sig) & (s_flat > 0)
    assert np.all(np.abs(sig[ok] - s_flat[ok]) <= 1e-13 * s_flat[ok])
    ref, st_ref, v, kap = _iv_ref(c)
    assert np.array_equal(st, st_ref)
    _check_sigma(sig, ref, st_ref, v, kap, tol_rest=1e-12, name="chains")
    # the direct launch (same kernel) reproduces the graph replay bit for bit
    plan.run_direct()
    assert np.array_equal(np.concatenate([_np(ch["sigma"]) for ch in chains]), sig, equal_nan=True)
    info = plan.info()
    assert info["quotes"] == c["offsets"][-1] and info["tiles"] > 0
    tune = plan.tuning()
    if autotune:
        assert tune["source"] in ("timed", "cached") and tune["best_ms"] > 0
    else:
        assert tune["source"] == "default" and (info["block"], info["quotes_per_thread"]) == (256, 4)
    plan.destroy()


def test_chains_every_launch_shape_and_the_cache_file(fv, torch_dev, tmp_path, monkeypatch):
    # Every compiled launch shape, forced through a seeded tuning-cache file,
    # gives the flat kernel's results; then a timed plan records its winner
    # in the file (FV_AUTOTUNE_CACHE), and FV_AUTOTUNE=0 overrides the argument.
    c = wl.fill_prices(wl.chains(40, seed=29, max_len=5000), orc.price_f64)
    chains = _chain_tensors(torch_dev, c)
    s_flat, st_flat = fv.fv_implied_vol(fv.FV_BLACK76, fv.FV_LBR,
                                        *_args(torch_dev, c, ("P", "S_or_F", "K", "T", "r")), None,
                                        _dev(torch_dev, c["flag"]))
    s_flat, st_flat = _np(s_flat), _np(st_flat)
    path = str(tmp_path / "tune.json")
    monkeypatch.setenv("FV_AUTOTUNE_CACHE", path)
    key = fv.fv_chains_plan_create(fv.FV_BLACK76, chains, autotune=False).tuning()["key"]
    assert key.count("|") == 5
    shapes = [(b, q) for b in (64, 128, 256, 512) for q in (1, 2, 4) if b * q <= 1024]
    for block, qpt in shapes:
        fv.fv_autotune_cache_put(path, key, block, qpt, 1, 1.0)
        plan = fv.fv_chains_plan_create(fv.FV_BLACK76, chains, autotune=True)
        info, tune = plan.info(), plan.tuning()
        assert tune["source"] == "cached" and tune["blocks_per_sm"] == 1
        assert (info["block"], info["quotes_per_thread"]) == (block, qpt)
        assert info["grid"] == min(info["tiles"], torch_dev[0].cuda.get_device_properties(0).multi_processor_count)
        for ch in chains:
            ch["sigma"].fill_(-7.0)
            ch["status"].fill_(9)
        plan.run()
        sig = np.concatenate([_np(ch["sigma"]) for ch in chains])
        st = np.concatenate([_np(ch["status"]) for ch in chains])
        assert np.array_equal(st, st_flat), (block, qpt)
        assert np.array_equal(np.isnan(sig), np.isnan(s_flat))
        ok = ~np.isnan(sig) & (s_flat > 0)
        assert np.all(np.abs(sig[ok] - s_flat[ok]) <= 1e-13 * s_flat[ok]), (block, qpt)
        plan.destroy()
    # an entry naming no compiled shape is ignored: the plan times the candidates
    fv.fv_autotune_cache_put(path, key, 96, 3, 1, 1.0)
    plan = fv.fv_chains_plan_create(fv.FV_BLACK76, chains, autotune=True)
    tune = plan.tuning()
    assert tune["source"] == "timed" and tune["candidates"] >= len(shapes)
    rec = fv.fv_autotune_cache_get(path, key)
    assert (rec["block"], rec["quotes_per_thread"], rec["blocks_per_sm"]) == (
        plan.info()["block"], plan.info()["quotes_per_thread"], tune["blocks_per_sm"])
    plan.destroy()
    monkeypatch.setenv("FV_AUTOTUNE", "0")
    assert fv.fv_chains_plan_create(fv.FV_BLACK76, chains, autotune=True).tuning()["source"] == "default"


def test_chains_with_empty_chains(fv, torch_dev):
    torch, dev = torch_dev
    c = wl.fill_prices(wl.chains(5, seed=11, max_len=100), orc.price)
    chains = _chain_tensors(torch_dev, c)
    e = lambda dt: torch.empty(0, dtype=dt, device=dev)
    chains.insert(2, dict(price=e(torch.float64), K=e(torch.float64), flag=e(torch.int8),
                          sigma=e(torch.float64), status=e(torch.uint8), S_or_F=100.0, T=1.0, r=0.0))
    plan = fv.fv_chains_plan_create(fv.FV_BLACK76, chains, autotune=False)
    plan.run()
    torch.cuda.synchronize()
    assert plan.info()["quotes"] == c["offsets"][-1]


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 255, 257, 4097])
def test_ragged_sizes_and_canaries(fv, torch_dev, n):
    torch, dev = torch_dev
    w = wl.fill_prices(wl.black76_quotes(n, seed=n), orc.price)
    ref, st_ref, v, kap = _iv_ref(w)
    pad = 64
    sig_buf = torch.full((n + 2 * pad,), 123.0, dtype=torch.float64, device=dev)
    st_buf = torch.full((n + 2 * pad,), 77, dtype=torch.uint8, device=dev)
    out_s, out_st = sig_buf[pad:pad + n], st_buf[pad:pad + n]
    P, F, K, T, r, _ = _args(torch_dev, w)
    fv.fv_implied_vol(fv.FV_BLACK76, fv.FV_LBR, P, F, K, T, r, None, _dev(torch_dev, w["flag"]),
                      out_s, out_st)
    sb, tb = _np(sig_buf), _np(st_buf)
    assert np.all(sb[:pad] == 123.0) and np.all(sb[pad + n:] == 123.0)
    assert np.all(tb[:pad] == 77) and np.all(tb[pad + n:] == 77)
    assert np.array_equal(tb[pad:pad + n], st_ref)
    _check_sigma(sb[pad:pad + n], ref, st_ref, v, kap, tol_rest=1e-12)


def test_misaligned_views(fv, torch_dev):
    # element offsets of 1 break 16-byte alignment of every array
    torch, dev = torch_dev
    n = 1000
    w = wl.fill_prices(wl.black76_quotes(n, seed=12), orc.price)
    ref, st_ref, v, kap = _iv_ref(w)

    def off(a, dt):
        t = torch.zeros(n + 1, dtype=dt, device=dev)
        t[1:] = torch.tensor(a, dtype=dt, device=dev)
        return t[1:]

    args = [off(w[k], torch.float64) for k in ("P", "S_or_F", "K", "T", "r")]
    s = off(np.zeros(n), torch.float64)
    st = off(np.zeros(n, np.uint8), torch.uint8)
    fv.fv_implied_vol(fv.FV_BLACK76, fv.FV_LBR, *args, None, off(w["flag"], torch.int8), s, st)
    assert np.array_equal(_np(st), st_ref)
    _check_sigma(_np(s), ref, st_ref, v, kap, tol_rest=1e-12)


def test_invalid_and_boundary_quotes(fv, torch_dev):
    nan, inf = float("nan"), float("inf")
    # (P, F, K, T, r, flag): r = 0 makes the bounds exact
    rows = [(10.0, 100, 90, 1, 0, 1), (10 * (1 - 1e-12), 100, 90, 1, 0, 1), (-1e-3, 100, 90, 1, 0, -1),
            (0.0, 100, 90, 1, 0, -1), (100.0, 100, 90, 1, 0, 1), (90.0, 100, 90, 1, 0, -1),
            (nan, 100, 90, 1, 0, 1), (5.0, 100, 90, 1, 0, 0), (5.0, 100, -90, 1, 0, 1),
            (5.0, 100, 90, 0, 0, 1), (5.0, inf, 90, 1, 0, 1), (5.0, 100, 90, 1, nan, 1),
            (12.0, 100, 90, 1, 0, 1), (3.0, 100, 100, 0.5, 0.0, -1), (1e-300, 100, 150, 0.1, 0.0, 1)]
    a = np.array(rows, dtype=np.float64)
    w = dict(model=0, P=a[:, 0], S_or_F=a[:, 1], K=a[:, 2], T=a[:, 3], r=a[:, 4], q=None,
             flag=a[:, 5].astype(np.int8))
    ref, st_ref, v, kap = _iv_ref(w)
    for solver in (fv.FV_LBR, fv.FV_HALLEY):
        s, st = fv.fv_implied_vol(0, solver, *_args(torch_dev, w), _dev(torch_dev, w["flag"]))
        assert np.array_equal(_np(st), st_ref)
        _check_sigma(_np(s), ref, st_ref, v, kap, tol_rest=1e-12)
    assert list(st_ref[:12]) == [0, 1, 1, 0, 2, 2, 3, 3, 3, 3, 3, 3]


def _status_edge_quotes():
    """Black-76 quotes (F = 100, T = 1, r = 0, so beta = P / sqrt(F K)) built
    in 50 digits at k units of 2^-52 from each threshold of the status rule
    (below intrinsic at iota (1 - e_s), at intrinsic at iota (1 + e_s), above
    the bound at b_max (1 - e_s) of the reduced quote, e_s = 64 * 2^-52), and
    the status and sigma class the rule's definition gives each side."""
    from decimal import Decimal, getcontext
    getcontext().prec = 50
    F, u = Decimal(100), Decimal(2) ** -52
    es = 64 * u
    P, K, flag, want, zero = [], [], [], [], []
    for k in (-48, -20, -6, 6, 20, 48):
        for Kv, fl, which in ((90, 1, "below"), (110, -1, "below"), (90, 1, "at"),
                              (110, 1, "above"), (90, -1, "above"), (90, 1, "above")):
            x = (F / Decimal(Kv)).ln()
            itm = fl * x > 0
            if which != "above" and not itm:
                continue
            a = abs(x) / 2
            iota = (a.exp() - (-a).exp()) if itm else Decimal(0)
            bmax = (-a).exp()
            if which == "below":
                beta = iota * (1 - es) * (1 + k * u)
                st, z = (orc.BELOW_INTRINSIC, False) if k < 0 else (orc.OK, True)
            elif which == "at":
                beta = iota * (1 + es) * (1 + k * u)
                st, z = orc.OK, k < 0
            else:
                beta = iota + bmax * (1 - es) * (1 + k * u)
                st, z = (orc.ABOVE_MAX, False) if k > 0 else (orc.OK, False)
            P.append(float(beta * (F * Decimal(Kv)).sqrt()))
            K.append(float(Kv))
            flag.append(fl)
            want.append(st)
            zero.append(z)
    return (np.array(P), np.array(K), np.array(flag, np.int8), np.array(want, np.uint8),
            np.array(zero))


def test_status_edges_on_every_path(fv, torch_dev):
    # Every solver decides the quotes 6 to 48 units of 2^-52 from a threshold
    # as the rule's definition (and the oracle's FP64 rule) does, in the small,
    # medium and large launch shapes: the double-float rule of the mixed and
    # FP32 tiles hands such quotes to the FP64 rule
    torch, dev = torch_dev
    P, K, flag, want, zero = _status_edge_quotes()
    st_o = orc.status(orc.BLACK76, P, np.full(P.size, 100.0), K, np.ones(P.size), np.zeros(P.size),
                      None, flag)[0]
    assert np.array_equal(st_o, want)
    for n in (P.size, 100000, 1 << 17):
        reps = -(-n // P.size)
        t = lambda a: torch.tensor(np.tile(a, reps)[:n], device=dev)
        args = [t(P), torch.full((n,), 100.0, dtype=torch.float64, device=dev), t(K),
                torch.ones(n, dtype=torch.float64, device=dev),
                torch.zeros(n, dtype=torch.float64, device=dev)]
        fl = t(flag)
        w, z = np.tile(want, reps)[:n], np.tile(zero, reps)[:n]
        for solver, prec in ((0, 0), (0, 1), (0, 2), (1, 0), (1, 2)):
            s, st = fv.fv_implied_vol_ex(fv.FV_BLACK76, solver, prec, *args, None, fl)
            s, st = _np(s), _np(st)
            assert np.array_equal(st, w), (n, solver, prec, int((st != w).sum()))
            ok = w == orc.OK
            assert np.all(s[ok & z] == 0.0), (n, solver, prec)
            if prec != 2:  # FP32 paths: only what the rule decides (beside the bound sigma may overflow)
                assert np.all(s[ok & ~z] > 0.0), (n, solver, prec)
            assert np.all(np.isnan(s[~ok])), (n, solver, prec)


def test_zero_length_is_a_noop(fv, torch_dev):
    torch, dev = torch_dev
    e = torch.empty(0, dtype=torch.float64, device=dev)
    s, st = fv.fv_implied_vol(0, 0, e, e, e, e, e, None, torch.empty(0, dtype=torch.int8, device=dev))
    assert s.numel() == 0 and st.numel() == 0


def test_abi_argument_errors(fv, torch_dev):
    lib = fv.library()
    torch, dev = torch_dev
    x = torch.ones(4, dtype=torch.float64, device=dev)
    p = ctypes.c_void_p(x.data_ptr())
    assert lib.fv_implied_vol(7, 0, p, p, p, p, p, None, p, 4, p, p, None) == fv.FV_ERR_ARG
    assert lib.fv_implied_vol(0, 5, p, p, p, p, p, None, p, 4, p, p, None) == fv.FV_ERR_ARG
    assert lib.fv_implied_vol(0, 0, p, p, p, p, p, None, p, -1, p, p, None) == fv.FV_ERR_ARG
    assert lib.fv_implied_vol(0, 0, None, p, p, p, p, None, p, 4, p, p, None) == fv.FV_ERR_ARG
    assert lib.fv_implied_vol(2, 0, p, p, p, p, p, None, p, 4, p, p, None) == fv.FV_ERR_ARG  # BSM needs q
    assert lib.fv_implied_vol_ex(0, 1, 1, 0, p, p, p, p, p, None, p, 4, p, p, None) == fv.FV_ERR_UNSUPPORTED
    assert lib.fv_implied_vol_ws(0, 1, p, p, p, p, p, None, p, 4, p, p, p, 8, None) == fv.FV_ERR_ARG
    assert b"workspace" in lib.fv_last_error()
    torch.cuda.synchronize()


# ---------------------------------------------------------------------------
# host-resident batches through the stream plan
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("solver,prec", [(0, 0), (0, 1), (0, 2), (1, 0)])
def test_host_streaming_matches_device(fv, torch_dev, solver, prec):
    # pinned host arrays: the direct mode (the solver reads and writes them in
    # place over the CPU-GPU link) runs the device call's kernel on the same
    # quotes, bit for bit; the staged mode (chunks of up to 100,000 quotes,
    # ramped at both ends, copied on two streams) solves its small chunks with
    # the unbinned kernel, equal within rounding
    torch, dev = torch_dev
    w = wl.fill_prices(wl.bsm_grid(1000, 300, seed=41), orc.price_f64)
    keys = ("P", "S_or_F", "K", "T", "r", "q", "flag")
    host = {k: torch.tensor(w[k]).pin_memory() for k in keys}
    s_d, st_d = fv.fv_implied_vol_ex(fv.FV_BSM, solver, prec, *_args(torch_dev, w),
                                     _dev(torch_dev, w["flag"]))
    s_d, st_d = _np(s_d), _np(st_d)
    plan = fv.fv_stream_plan_create(100000)
    assert plan.last_transfer == fv.FV_TRANSFER_AUTO
    for mode, taken in ((fv.FV_TRANSFER_AUTO, fv.FV_TRANSFER_DIRECT),
                        (fv.FV_TRANSFER_STAGED, fv.FV_TRANSFER_STAGED),
                        (fv.FV_TRANSFER_DIRECT, fv.FV_TRANSFER_DIRECT)):
        plan.set_transfer(mode)
        s_h, st_h = plan.implied_vol(fv.FV_BSM, solver, prec, *[host[k] for k in keys])
        torch.cuda.synchronize()
        assert plan.last_transfer == taken
        s_h, st_h = s_h.numpy(), st_h.numpy()
        assert np.array_equal(st_h, st_d), mode
        assert np.array_equal(np.isnan(s_h), np.isnan(s_d)), mode
        ok = ~np.isnan(s_d) & (s_d > 0)
        if taken == fv.FV_TRANSFER_DIRECT:
            assert np.array_equal(s_h[ok], s_d[ok]), mode
        elif prec != fv.FV_FP32:  # FP32: rounding differs by the conditioning
            assert np.all(np.abs(s_h[ok] - s_d[ok]) <= 1e-12 * s_d[ok]), mode
    # pageable arrays: AUTO stages them, DIRECT refuses them before any work
    pageable = {k: torch.tensor(w[k]) for k in keys}
    assert not pageable["P"].is_pinned()
    plan.set_transfer(fv.FV_TRANSFER_DIRECT)
    with pytest.raises(fv.FvError) as e:
        plan.implied_vol(fv.FV_BSM, solver, prec, *[pageable[k] for k in keys])
    assert e.value.code == fv.FV_ERR_ARG
    plan.set_transfer(fv.FV_TRANSFER_AUTO)
    s_p, st_p = plan.implied_vol(fv.FV_BSM, solver, prec, *[pageable[k] for k in keys],
                                 out_sigma=torch.empty(s_d.size, dtype=torch.float64),
                                 status=torch.empty(s_d.size, dtype=torch.uint8))
    torch.cuda.synchronize()
    assert plan.last_transfer == fv.FV_TRANSFER_STAGED
    assert np.array_equal(st_p.numpy(), st_d)
    with pytest.raises(fv.FvError) as e:
        plan.set_transfer(7)
    assert e.value.code == fv.FV_ERR_ARG
    plan.destroy()


def test_host_batches_with_fp32_inputs(fv, torch_dev):
    # FP32 host arrays through the stream plan: read in place (direct) they give
    # the device call's results bit for bit; copied in chunks (staged) the same
    # statuses and, in FP64 and mixed, sigma within rounding
    torch, dev = torch_dev
    w = wl.black76_fp32(200000, seed=12)
    wl.fill_prices(w, orc.price, price_dtype=np.float32)
    keys = ("P", "S_or_F", "K", "T", "r")
    host = {k: torch.tensor(w[k]).pin_memory() for k in keys}
    hflag = torch.tensor(w["flag"]).pin_memory()
    devs = [torch.tensor(w[k], device=dev) for k in keys]
    dflag = _dev(torch_dev, w["flag"])
    plan = fv.fv_stream_plan_create(50000)
    for prec in (fv.FV_FP64, fv.FV_MIXED, fv.FV_FP32):
        s_d, st_d = fv.fv_implied_vol_ex(fv.FV_BLACK76, fv.FV_LBR, prec, *devs, None, dflag)
        s_d, st_d = _np(s_d), _np(st_d)
        for mode in (fv.FV_TRANSFER_DIRECT, fv.FV_TRANSFER_STAGED):
            plan.set_transfer(mode)
            s_h, st_h = plan.implied_vol(fv.FV_BLACK76, fv.FV_LBR, prec, *[host[k] for k in keys],
                                         None, hflag)
            torch.cuda.synchronize()
            assert plan.last_transfer == mode
            s_h, st_h = s_h.numpy(), st_h.numpy()
            assert np.array_equal(st_h, st_d), (prec, mode)
            assert np.array_equal(np.isnan(s_h), np.isnan(s_d)), (prec, mode)
            ok = ~np.isnan(s_d) & (s_d > 0)
            if mode == fv.FV_TRANSFER_DIRECT:
                assert np.array_equal(s_h[ok], s_d[ok]), prec
            elif prec != fv.FV_FP32:
                assert np.all(np.abs(s_h[ok] - s_d[ok]) <= 1e-12 * s_d[ok]), prec
    plan.destroy()


# ---------------------------------------------------------------------------
# the implied-volatility calls allocate nothing and never synchronise
# ---------------------------------------------------------------------------
def test_iv_calls_capture_into_a_graph(fv, torch_dev):
    # Each solver captures into a CUDA graph on a side stream in the global
    # capture mode, which fails on any synchronising or allocating call from
    # any thread; the batch (1,433,600 quotes, dynamic tiles with their
    # counter memset) is larger than every Halley call before it in this module.
    # Replays reproduce the direct call bit for bit, also after the outputs
    # (which hold the tile counters while a call runs) were overwritten.
    torch, dev = torch_dev
    w = wl.fill_prices(wl.bsm_grid(2048, 700, seed=43), orc.price_f64)
    args = _args(torch_dev, w)
    flag = _dev(torch_dev, w["flag"])
    n = flag.numel()
    for solver, prec in ((fv.FV_HALLEY, fv.FV_FP64), (fv.FV_HALLEY, fv.FV_FP32),
                         (fv.FV_LBR, fv.FV_FP64), (fv.FV_LBR, fv.FV_MIXED)):
        out = torch.full((n,), -1.0, dtype=torch.float64, device=dev)
        st = torch.full((n,), 9, dtype=torch.uint8, device=dev)
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=side, capture_error_mode="global"):
            fv.fv_implied_vol_ex(fv.FV_BSM, solver, prec, *args, flag, out, st)
        torch.cuda.synchronize()
        s_ref, st_ref = fv.fv_implied_vol_ex(fv.FV_BSM, solver, prec, *args, flag)
        for fill in (-1.0, 3.0):
            out.fill_(fill)
            st.fill_(9)
            g.replay()
            torch.cuda.synchronize()
            assert torch.equal(st, st_ref), (solver, prec)
            assert torch.equal(out.nan_to_num(-7.0), s_ref.nan_to_num(-7.0)), (solver, prec)
        del g
    _sampled_parity(fv, torch_dev, w, _np(s_ref), _np(st_ref), fv.FV_BSM, n_sample=2048, seed=8)


def test_halley_workspace_and_tiled_arrangements_agree(fv, torch_dev):
    # fv_implied_vol_ws compacts the failures into a device list and runs the
    # fallback as a second kernel; fv_implied_vol compacts them per tile in
    # shared memory.  Same per-quote arithmetic, same results, on a batch
    # where both the static (small) and dynamic (large) tilings run.
    torch, dev = torch_dev
    for n_s, n_m in ((300, 100), (1024, 300)):
        w = wl.fill_prices(wl.bsm_grid(n_s, n_m, seed=44), orc.price_f64)
        args = _args(torch_dev, w)
        flag = _dev(torch_dev, w["flag"])
        n = flag.numel()
        ws = torch.zeros(fv.fv_workspace_size(fv.FV_HALLEY, n), dtype=torch.uint8, device=dev)
        s_ws, st_ws = fv.fv_implied_vol_ws(fv.FV_BSM, fv.FV_HALLEY, *args, flag, ws)
        torch.cuda.synchronize()
        n_fallback = int(ws[:4].cpu().numpy().view(np.uint32)[0])
        s_t, st_t = fv.fv_implied_vol(fv.FV_BSM, fv.FV_HALLEY, *args, flag)
        assert torch.equal(st_ws, st_t)
        a, b = _np(s_ws), _np(s_t)
        assert np.array_equal(np.isnan(a), np.isnan(b))
        ok = ~np.isnan(b) & (b > 0)
        # the compiler may contract the same source into FMAs differently in
        # the two kernels: only rounding, amplified by the conditioning, differs
        rel = np.abs(a[ok] - b[ok]) / b[ok]
        assert rel.max() <= 1e-12, rel.max()
        # the grid's wings fail the sweeps' convergence test: the fallback runs
        assert 0 < n_fallback < n


# ---------------------------------------------------------------------------
# binned (large batches) and unbinned (small batches) kernels agree
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_binned_matches_unbinned_and_oracle(fv, torch_dev, prec):
    # 2^18 quotes run the region-binned kernel, their first 2^16 alone the
    # unbinned one: the same arithmetic per quote, so equal within rounding
    w = wl.fill_prices(wl.bsm_grid(4096, 64, seed=21), orc.price_f64)
    args = _args(torch_dev, w)
    flag = _dev(torch_dev, w["flag"])
    p = fv.FV_FP64 if prec == "fp64" else fv.FV_MIXED
    s_big, st_big = fv.fv_implied_vol_ex(fv.FV_BSM, fv.FV_LBR, p, *args, flag)
    m = 1 << 16
    s_small, st_small = fv.fv_implied_vol_ex(fv.FV_BSM, fv.FV_LBR, p, *[a[:m] for a in args],
                                             flag[:m])
    s_big, st_big, s_small = _np(s_big), _np(st_big), _np(s_small)
    assert np.array_equal(st_big[:m], _np(st_small))
    a, b = s_big[:m], s_small
    assert np.array_equal(np.isnan(a), np.isnan(b))
    ok = ~np.isnan(b) & (b > 0)
    assert np.all(np.abs(a[ok] - b[ok]) <= 1e-12 * b[ok])
    _sampled_parity(fv, torch_dev, w, s_big, st_big, fv.FV_BSM, n_sample=4096, seed=3)


# medium batches (from 98,304 quotes in FP64, 65,536 in mixed and FP32, up to
# 2^17): 128-quote binned tiles, one per block, refining their ill-conditioned
# quotes in the tile instead of a second kernel
MID_SIZES = {"fp64": (98304, 100000, 131071), "mixed": (65536, 100000, 131071),
             "fp32": (65536, 100000, 131071)}


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("workload", ["black76", "grid"])
def test_medium_batches_match_large_and_oracle(fv, torch_dev, prec, workload):
    # the first m quotes of a 2^18-quote call, solved alone by the medium-batch
    # kernel: the same per-quote arithmetic as the large-batch kernel and its
    # refinement pass, so equal within rounding; then against the definition.
    # The Black-76 quotes alternate flags: half are in the money, and a few
    # per cent of those need the double-double reduced price
    n = 1 << 18
    if workload == "black76":
        w = wl.fill_prices(wl.black76_quotes(n, seed=23), orc.price_f64)
        model = fv.FV_BLACK76
        _, x, beta, _ = orc.status(model, w["P"], w["S_or_F"], w["K"], w["T"], w["r"], None,
                                   w["flag"])
        iota = np.maximum(w["flag"] * (np.exp(x / 2) - np.exp(-x / 2)), 0.0)
        assert ((iota > 0) & (beta - iota < beta / 64)).sum() > 100  # the in-tile refinement runs
    else:
        w = wl.fill_prices(wl.bsm_grid(4096, 64, seed=22), orc.price_f64)
        model = fv.FV_BSM
    args = _args(torch_dev, w)
    flag = _dev(torch_dev, w["flag"])
    p = {"fp64": fv.FV_FP64, "mixed": fv.FV_MIXED, "fp32": fv.FV_FP32}[prec]
    s_big, st_big = fv.fv_implied_vol_ex(model, fv.FV_LBR, p, *args, flag)
    s_big, st_big = _np(s_big), _np(st_big)
    for m in MID_SIZES[prec]:
        s_m, st_m = fv.fv_implied_vol_ex(model, fv.FV_LBR, p, *[None if a is None else a[:m]
                                                                 for a in args], flag[:m])
        s_m, st_m = _np(s_m), _np(st_m)
        assert np.array_equal(st_big[:m], st_m), m
        a, b = s_big[:m], s_m
        assert np.array_equal(np.isnan(a), np.isnan(b)), m
        ok = ~np.isnan(b) & (b > 0)
        if prec == "fp32":  # the same double-float tile: rounding aside, equal
            assert np.mean(a[ok] == b[ok]) > 0.999, m
        else:
            assert np.all(np.abs(a[ok] - b[ok]) <= 1e-12 * b[ok]), m
    sub = {k: (None if w.get(k) is None else np.asarray(w[k])[:m]) for k in
           ("P", "S_or_F", "K", "T", "r", "q", "flag")}
    _sampled_parity(fv, torch_dev, sub, s_m, st_m, model, n_sample=8192, seed=4,
                    tol_gate=1e-5 if prec == "fp32" else 1e-12)


# ---------------------------------------------------------------------------
# full reference sizes, in the launch configuration the benchmark times
# ---------------------------------------------------------------------------
def _status_parity(st, w, model, max_ambiguous=1e-3, max_flipped=1e-6):
    """Status bit-identical to the oracle's FP64 rule for every quote whose
    decision quantities are more than 16 ulp from a threshold; within 16 ulp a
    one-ulp difference between two libm implementations of exp/log1p/expm1 can
    flip the decision, so there the status must only be one of the two
    neighbours of the threshold.  Returns the mask of unambiguous quotes."""
    st_all, _, _, margin = orc.status(model, w["P"], w["S_or_F"], w["K"], w["T"], w["r"],
                                      w.get("q"), w["flag"])
    amb = margin <= 16.0
    clear = ~amb
    assert np.array_equal(st[clear], st_all[clear])
    assert amb.mean() <= max_ambiguous, "ambiguous fraction %g" % amb.mean()
    assert np.all(np.isin(st[amb], (orc.OK, orc.BELOW_INTRINSIC, orc.ABOVE_MAX)))
    flipped = (st != st_all).sum()
    assert flipped <= max_flipped * st.size, "%d of %d statuses differ" % (flipped, st.size)
    return clear & (st == st_all)


def _sampled_parity(fv, torch_dev, w, sig, st, model, n_sample=2048, seed=0, tol_gate=1e-12):
    clear = _status_parity(st, w, model)
    g = np.random.default_rng(seed)
    pool = np.nonzero(clear)[0]
    idx = np.sort(g.choice(pool, size=min(n_sample, pool.size), replace=False))
    sub = {k: (None if w.get(k) is None else np.asarray(w[k])[idx]) for k in
           ("P", "S_or_F", "K", "T", "r", "q", "flag")}
    sub["model"] = model
    ref, st_ref, v, kap = _iv_ref(sub)
    assert np.array_equal(st[idx], st_ref)
    _check_sigma(sig[idx], ref, st_ref, v, kap, tol_gate=tol_gate,
                 tol_rest=1e-12 if tol_gate <= 1e-12 else None)


@pytest.fixture(scope="module")
def full_grid():
    """The 16,777,216-quote BSM grid the benchmark times, priced in binary128,
    with the oracle's status rule for every quote, the oracle's step-by-step
    FP64 LBR for every quote, and the definition (binary128 root) on 262,144
    quotes sampled among those clear of a status threshold."""
    w = wl.fill_prices(wl.bsm_grid(4096, 4096, seed=1), orc.price)
    keys = ("P", "S_or_F", "K", "T", "r", "q", "flag")
    st_all, _, beta, margin = orc.status(wl.BSM, *[w[k] for k in keys])
    lbr, st_lbr, _ = orc.iv_lbr(wl.BSM, *[w[k] for k in keys], n_iter=3)
    g = np.random.default_rng(17)
    idx = np.sort(g.choice(np.nonzero(margin > 16.0)[0], size=262144, replace=False))
    sub = {k: np.asarray(w[k])[idx] for k in keys}
    sub["model"] = wl.BSM
    return dict(w=w, st=st_all, beta=beta, margin=margin, lbr=lbr, st_lbr=st_lbr, idx=idx,
                ref=_iv_ref(sub))


# (solver, precision, gated tolerance, conditioning bound) of every path the
# benchmark times on the grid
FULL_PATHS = {"lbr": (0, 0, 1e-12, 1e-12), "mixed": (0, 1, 1e-12, 1e-12),
              "halley": (1, 0, 1e-12, 1e-12), "fp32": (0, 2, 1e-5, None),
              "halley32": (1, 2, 1e-4, None)}


@pytest.mark.parametrize("path", list(FULL_PATHS))
def test_full_size_bsm_grid(fv, torch_dev, full_grid, path):
    # the launch configuration of the benchmark: one call over the whole grid
    solver, prec, tol, tol_rest = FULL_PATHS[path]
    w = full_grid["w"]
    s, st = fv.fv_implied_vol_ex(fv.FV_BSM, solver, prec, *_args(torch_dev, w),
                                 _dev(torch_dev, w["flag"]))
    s, st = _np(s), _np(st)
    # status: bit-identical for every quote (binary128 prices keep every quote
    # clear of the rule's thresholds)
    assert np.array_equal(st, full_grid["st"]), "%d statuses differ" % (st != full_grid["st"]).sum()
    # sigma against the definition on the sampled quotes
    idx = full_grid["idx"]
    ref, st_ref, v, kap = full_grid["ref"]
    assert np.array_equal(st[idx], st_ref)
    _check_sigma(s[idx], ref, st_ref, v, kap, tol_gate=tol, tol_rest=tol_rest, name=path)
    if tol_rest is None:
        return
    # every quote against the oracle's FP64 LBR (within 4 eps (1 + kappa) of
    # the definition, a pin of the oracle): the two may differ by both
    # errors, so the bound is 1e-12 + 16 eps (1 + kappa) with kappa from the
    # oracle at its own sigma.  The oracle's FP64 LBR works on beta itself,
    # so it covers the quotes whose normalised price is a normal FP64 number
    # (beta >= 1e-290); below it (prices at the bottom of the FP64 range,
    # ~6 % of the grid, most of them 0) the sampled comparison with the
    # definition above applies, and a zero price must give sigma = 0.
    lbr = full_grid["lbr"]
    assert np.array_equal(full_grid["st_lbr"], full_grid["st"])
    assert np.all(np.isnan(s[st != orc.OK])), path
    assert np.all(s[(st == orc.OK) & (w["P"] == 0)] == 0.0), path
    normal = (st == orc.OK) & (full_grid["beta"] >= 1e-290)
    assert np.all(s[normal & (lbr == 0)] == 0.0), path
    solved = normal & (lbr > 0)
    assert solved.sum() > 0.9 * (st == orc.OK).sum()
    keys = ("P", "S_or_F", "K", "T", "r", "q", "flag")
    v_all, kap_all = orc.conditioning(wl.BSM, *[w[k] for k in keys], lbr)
    rel = np.abs(s[solved] - lbr[solved]) / lbr[solved]
    k = np.nan_to_num(kap_all[solved], nan=np.inf, posinf=np.inf)
    bound = 1e-12 + 16 * EPS * (1 + k)
    bad = rel > bound
    assert not bad.any(), "%s: %d of %d quotes beyond the bound (worst %.3g)" % (
        path, bad.sum(), solved.sum(), rel[bad].max())
    gate = (v_all[solved] > 1e-8) & (k <= 1e3)
    assert rel[gate].max() <= 2e-12, "%s: gated max rel %.3g vs the oracle's LBR" % (
        path, rel[gate].max())


def test_full_size_fp32_inputs_mixed(fv, torch_dev):
    torch, dev = torch_dev
    w = wl.black76_fp32(67108864, seed=2)
    wl.fill_prices(w, orc.price, price_dtype=np.float32)
    args = [torch.tensor(w[k], device=dev) for k in ("P", "S_or_F", "K", "T", "r")]
    flag = _dev(torch_dev, w["flag"])
    s, st = fv.fv_implied_vol_ex(fv.FV_BLACK76, fv.FV_LBR, fv.FV_MIXED, *args, None, flag)
    w64 = {k: (None if w.get(k) is None else np.asarray(w[k], dtype=np.float64) if k != "flag"
               else w[k]) for k in ("P", "S_or_F", "K", "T", "r", "q", "flag")}
    _sampled_parity(fv, torch_dev, w64, _np(s), _np(st), fv.FV_BLACK76, n_sample=65536)


def test_full_size_chains(fv, torch_dev):
    # 10,000 chains (72.8 M quotes), the plan tuned on them (every shape timed)
    c = wl.fill_prices(wl.chains(10000, seed=3), orc.price)
    chains = _chain_tensors(torch_dev, c)
    plan = fv.fv_chains_plan_create(fv.FV_BLACK76, chains, autotune=True)
    assert plan.tuning()["source"] in ("timed", "cached")
    for ch in chains:
        ch["sigma"].fill_(-7.0)
        ch["status"].fill_(9)
    plan.run()
    sig = np.concatenate([_np(ch["sigma"]) for ch in chains])
    st = np.concatenate([_np(ch["status"]) for ch in chains])
    _sampled_parity(fv, torch_dev, c, sig, st, fv.FV_BLACK76, n_sample=65536)
    plan.destroy()


def test_full_size_adjoint(fv, torch_dev):
    w = wl.fill_prices(wl.bsm_quotes(8388608, seed=4), orc.price)
    ins = _args(torch_dev, w)
    flag = _dev(torch_dev, w["flag"])
    s, st = fv.fv_implied_vol(fv.FV_BSM, fv.FV_LBR, *ins, flag)
    adj = fv.fv_iv_adjoint(fv.FV_BSM, *ins, flag, s, st, _dev(torch_dev, w["grad_sigma"]))
    s_np, st_np = _np(s), _np(st)
    idx = np.random.default_rng(5).choice(s_np.size, 65536, replace=False)
    sub = lambda k: np.asarray(w[k])[idx]
    refs = orc.iv_grad(2, sub("S_or_F"), sub("K"), sub("T"), sub("r"), sub("q"), sub("flag"),
                       s_np[idx], st_np[idx], sub("grad_sigma"))
    v, kap = orc.conditioning(2, sub("P"), sub("S_or_F"), sub("K"), sub("T"), sub("r"), sub("q"),
                              sub("flag"), s_np[idx])
    ok = (st_np[idx] == 0) & (s_np[idx] > 0) & (v > 1e-8)
    for name, ref in zip(("P", "S", "K", "T", "r", "q"), refs):
        g = _np(adj[name])[idx]
        assert (np.abs(g[ok] - ref[ok]) / np.maximum(np.abs(ref[ok]), 1e-300)).max() <= 1e-11, name
