"""Pins of the CPU oracle against what the mathematics and the paper fix.

Every test here runs on the CPU.  None re-types the oracle's own formula: the
price is checked against the risk-neutral expectation by quadrature, the
normalised Black function against the closed form at the money and its series
limits, the implied volatility against an independent mpmath root and against
the closed-form inverse at the money, and the solvers of Section 2.2 against
the binary128 definition.
"""
import json
import math
import os

import mpmath as mp
import numpy as np
import pytest
from scipy import special

from oracle import oracle as orc
from paper_2604_27210_gb300 import workloads as wl

EPS = 2.0 ** -52
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# price and normalised Black
# ---------------------------------------------------------------------------
def _expectation_price(model, SF, K, T, r, q, sigma, theta):
    """Discounted E[(theta (F_T - K))^+] by quadrature over the lognormal law."""
    mp.mp.dps = 40
    SF, K, T, r, q, sigma = (mp.mpf(v) for v in (SF, K, T, r, q, sigma))
    F = SF if model == orc.BLACK76 else SF * mp.exp((r - q) * T)
    s = sigma * mp.sqrt(T)
    zk = (mp.log(K / F) + s * s / 2) / s  # F_T = K at z = zk

    def payoff(z):
        FT = F * mp.exp(-s * s / 2 + s * z)
        return max(theta * (FT - K), 0) * mp.npdf(z)

    lim = [-mp.inf, zk, mp.inf]
    return mp.exp(-r * T) * mp.quad(payoff, lim)


@pytest.mark.parametrize("model", [orc.BLACK76, orc.BLACK_SCHOLES, orc.BSM])
def test_price_equals_risk_neutral_expectation(model):
    cases = [(100.0, 95.0, 0.25, 0.05, 0.02, 0.2, 1), (100.0, 105.0, 0.25, 0.05, 0.02, 0.2, -1),
             (100.0, 130.0, 1.5, 0.01, 0.03, 0.35, 1), (100.0, 70.0, 0.1, 0.04, 0.0, 0.6, -1),
             (42.0, 40.0, 0.5, 0.1, 0.01, 0.2, 1), (100.0, 100.0, 2.0, 0.0, 0.0, 1.2, -1)]
    for SF, K, T, r, q, sig, th in cases:
        got = orc.price(model, SF, K, T, r, q, sig, th)[0]
        want = float(_expectation_price(model, SF, K, T, r, q if model == orc.BSM else 0.0, sig, th))
        assert got == pytest.approx(want, rel=1e-13, abs=1e-300)


def test_fp64_textbook_price_agrees_with_binary128():
    w = wl.bsm_quotes(20000, seed=13)
    for model in (orc.BLACK76, orc.BSM):
        a = orc.price_f64(model, w["S_or_F"], w["K"], w["T"], w["r"], w["q"], w["sigma_true"], w["flag"])
        b = orc.price(model, w["S_or_F"], w["K"], w["T"], w["r"], w["q"], w["sigma_true"], w["flag"])
        m = b > 1e-3  # away from the cancellation of deep out-of-the-money quotes
        assert (np.abs(a[m] - b[m]) / b[m]).max() <= 1e-12


def test_put_call_parity():
    w = wl.black76_quotes(512, seed=11)
    for model in (orc.BLACK76, orc.BSM):
        q = np.full(512, 0.02) if model == orc.BSM else None
        c = orc.price(model, w["S_or_F"], w["K"], w["T"], w["r"], q, w["sigma_true"], 1)
        p = orc.price(model, w["S_or_F"], w["K"], w["T"], w["r"], q, w["sigma_true"], -1)
        D = np.exp(-w["r"] * w["T"])
        F = w["S_or_F"] if model == orc.BLACK76 else w["S_or_F"] * np.exp((w["r"] - 0.02) * w["T"])
        np.testing.assert_allclose(c - p, D * (F - w["K"]), rtol=0, atol=1e-12 * 100)


def test_erfcx_against_mpmath():
    # erfcx(z) = exp(z^2) erfc(z), the function of the erfcx branch of Section 2.2
    g = np.random.default_rng(3)
    z = np.concatenate([g.uniform(-26.5, 0, 200), g.uniform(0, 8, 200),
                        np.exp(g.uniform(np.log(8), np.log(1e300), 200)), [0.0, 99.99, 100.0, 100.01]])
    got = orc.erfcx(z)
    mp.mp.dps = 40
    for zi, gi in zip(z, got):
        y = mp.mpf(zi)
        if y > 1e6:  # mpmath's erfc does not reach there: series to 1/z^6 (error < 1e-36)
            ref = (1 - 1 / (2 * y * y) + 3 / (4 * y ** 4)) / (y * mp.sqrt(mp.pi))
        else:
            ref = mp.exp(y ** 2) * mp.erfc(y)
        assert abs(float((gi - ref) / ref)) <= 2.0 ** -53 * 1.0001, zi
    sp = orc.erfcx(np.array([np.inf, -np.inf, -27.0, np.nan]))
    assert sp[0] == 0 and sp[1] == np.inf and sp[2] == np.inf and np.isnan(sp[3])


def test_normalised_black_at_the_money_is_erf():
    # x = 0: b(0, s) = Phi(s/2) - Phi(-s/2) = erf(s / (2 sqrt 2))
    s = np.logspace(-6, 1.3, 200)
    b = orc.normalised_black(np.zeros_like(s), s, 1)
    np.testing.assert_allclose(b, special.erf(s / (2 * math.sqrt(2))), rtol=4 * EPS, atol=0)


def test_normalised_black_brenner_subrahmanyam_limit():
    # at the money, b = s/sqrt(2 pi) - s^3/(24 sqrt(2 pi)) + O(s^5)
    s = np.array([1e-8, 1e-6, 1e-4, 1e-3])
    b = orc.normalised_black(np.zeros_like(s), s, 1)
    bs = s / math.sqrt(2 * math.pi) * (1 - s * s / 24)
    np.testing.assert_allclose(b, bs, rtol=1e-12)


def test_normalised_black_symmetries():
    g = np.random.default_rng(5)
    x = g.uniform(-4, 4, 300)
    s = np.exp(g.uniform(np.log(1e-3), np.log(5), 300))
    bc = orc.normalised_black(x, s, 1)
    bp = orc.normalised_black(x, s, -1)
    # call - put = e^{x/2} - e^{-x/2}
    assert np.all(np.abs((bc - bp) - 2 * np.sinh(x / 2)) <= 8 * EPS * np.exp(np.abs(x) / 2))
    # b(x, s, theta) = b(-x, s, -theta)
    np.testing.assert_allclose(bc, orc.normalised_black(-x, s, -1), rtol=8 * EPS, atol=1e-300)


def test_normalised_black_limits_and_monotonicity():
    for x in (-3.0, -0.2, 0.0):
        s = np.logspace(-3, 2, 400)
        b = orc.normalised_black(np.full_like(s, x), s, 1)
        assert np.all(np.diff(b) >= 0)
        assert b[-1] == pytest.approx(math.exp(x / 2), rel=1e-15)
    # s -> 0: the call tends to its intrinsic value max(e^{x/2}-e^{-x/2}, 0)
    assert orc.normalised_black(np.array([0.7]), np.array([1e-4]), 1)[0] == pytest.approx(
        2 * math.sinh(0.35), rel=1e-15)


# ---------------------------------------------------------------------------
# implied volatility by definition
# ---------------------------------------------------------------------------
def _gate(model, P, w, sig):
    v, kap = orc.conditioning(model, P, w["S_or_F"], w["K"], w["T"], w["r"], w.get("q"), w["flag"],
                              sig)
    return v, kap


def test_iv_round_trip_black76():
    w = wl.fill_prices(wl.black76_quotes(2048, seed=0), orc.price)
    sig, st = orc.iv(w["model"], w["P"], w["S_or_F"], w["K"], w["T"], w["r"], None, w["flag"])
    assert np.all(st == orc.OK)
    v, kap = _gate(w["model"], w["P"], w, sig)
    ok = sig > 0
    # the price was rounded to FP64: sigma moves by at most ~eps * kappa
    rel = np.abs(sig[ok] - w["sigma_true"][ok]) / w["sigma_true"][ok]
    assert np.all(rel <= 2 * EPS * (1 + kap[ok]))
    # price(iv(P)) == P within rounding where the normalised vega is not tiny
    back = orc.price(w["model"], w["S_or_F"], w["K"], w["T"], w["r"], None, sig, w["flag"])
    m = ok & (v > 1e-8)
    np.testing.assert_allclose(back[m], w["P"][m], rtol=1e-15)


def test_iv_at_the_money_closed_form():
    # x = 0: beta = erf(s / (2 sqrt 2))  =>  s = 2 sqrt(2) erfinv(beta)
    beta = np.linspace(1e-6, 0.99, 64)
    n = beta.size
    sig, st = orc.iv(orc.BLACK76, beta, np.ones(n), np.ones(n), np.ones(n), np.zeros(n), None,
                     np.ones(n, np.int8))
    mp.mp.dps = 40
    want = np.array([float(2 * mp.sqrt(2) * mp.erfinv(mp.mpf(b))) for b in beta])
    np.testing.assert_allclose(sig, want, rtol=2 * EPS)


def test_iv_matches_independent_high_precision_root():
    # brute force on tiny inputs: mpmath root of the textbook price at 40 digits
    w = wl.fill_prices(wl.bsm_grid(8, 4, seed=9, below_fraction=0.0), orc.price)
    sig, st = orc.iv(w["model"], w["P"], w["S_or_F"], w["K"], w["T"], w["r"], w["q"], w["flag"])
    mp.mp.dps = 40
    checked = 0
    for i in range(sig.size):
        if st[i] != orc.OK or not sig[i] > 0:
            continue
        S, K, T, r, q, th = (mp.mpf(float(w[k][i])) for k in ("S_or_F", "K", "T", "r", "q", "flag"))
        P = mp.mpf(float(w["P"][i]))

        def f(sg):
            s = sg * mp.sqrt(T)
            d1 = (mp.log(S / K) + (r - q + sg * sg / 2) * T) / s
            d2 = d1 - s
            V = th * (S * mp.exp(-q * T) * mp.ncdf(th * d1) - K * mp.exp(-r * T) * mp.ncdf(th * d2))
            return mp.log(V / P)  # relative residual: deep-wing prices reach 1e-200

        root = mp.findroot(f, (mp.mpf(float(sig[i])) * (1 - mp.mpf(10) ** -6),
                               mp.mpf(float(sig[i])) * (1 + mp.mpf(10) ** -6)), solver="anderson")
        assert float(root) == pytest.approx(sig[i], rel=4 * EPS), i
        checked += 1
    assert checked >= 16


def test_iv_put_call_parity_consistency():
    w = wl.fill_prices(wl.black76_quotes(512, seed=3), orc.price)
    th = w["flag"]
    D = np.exp(-w["r"] * w["T"])
    # the same option seen from the other side through put-call parity
    P_other = w["P"] - th * D * (w["S_or_F"] - w["K"])
    s1, st1 = orc.iv(0, w["P"], w["S_or_F"], w["K"], w["T"], w["r"], None, th)
    s2, st2 = orc.iv(0, P_other, w["S_or_F"], w["K"], w["T"], w["r"], None, -th)
    ok = (st1 == 0) & (st2 == 0) & (s1 > 0) & (s2 > 0)
    assert ok.sum() > 400
    v, kap = _gate(0, np.maximum(w["P"], P_other), w, s1)
    rel = np.abs(s1[ok] - s2[ok]) / s1[ok]
    assert np.all(rel <= 8 * EPS * (1 + kap[ok]))


def test_iv_power_of_two_scale_invariance():
    w = wl.fill_prices(wl.black76_quotes(256, seed=4), orc.price)
    s0, st0 = orc.iv(0, w["P"], w["S_or_F"], w["K"], w["T"], w["r"], None, w["flag"])
    for k in (-3, 2, 5):
        f = 4.0 ** k
        s1, st1 = orc.iv(0, w["P"] * f, w["S_or_F"] * f, w["K"] * f, w["T"], w["r"], None, w["flag"])
        assert np.array_equal(st0, st1)
        assert np.array_equal(s0, s1, equal_nan=True)


def test_iv_monotone_in_price():
    P = np.linspace(0.5, 20.0, 200)
    n = P.size
    sig, st = orc.iv(0, P, np.full(n, 100.0), np.full(n, 110.0), np.full(n, 0.7), np.full(n, 0.02),
                     None, np.ones(n, np.int8))
    assert np.all(st == 0) and np.all(np.diff(sig) > 0)


def test_status_decisions_at_exact_bounds():
    # r = 0 so discounting is exact: intrinsic = max(theta (F - K), 0), max = F (call) / K (put)
    F, K, T = 100.0, 90.0, 1.0
    cases = [  # (P, flag, expected status, expected sigma)
        (10.0, 1, orc.OK, 0.0),                      # exactly intrinsic -> sigma = 0
        (10.0 * (1 - 1e-12), 1, orc.BELOW_INTRINSIC, None),
        (-1e-3, -1, orc.BELOW_INTRINSIC, None),      # negative price of an OTM put
        (0.0, -1, orc.OK, 0.0),                      # zero price of an OTM put
        (100.0, 1, orc.ABOVE_MAX, None),             # call worth the forward
        (90.0, -1, orc.ABOVE_MAX, None),             # put worth the strike
        (150.0, 1, orc.ABOVE_MAX, None),
        (float("nan"), 1, orc.INVALID, None),
        (5.0, 0, orc.INVALID, None),                 # flag neither +1 nor -1
        (12.0, 1, orc.OK, "positive"),
    ]
    for P, fl, want_st, want_sig in cases:
        sig, st = orc.iv(0, P, F, K, T, 0.0, None, fl)
        assert st[0] == want_st, (P, fl)
        if want_sig is None:
            assert math.isnan(sig[0])
        elif want_sig == "positive":
            assert sig[0] > 0
        else:
            assert sig[0] == want_sig
    bad = [dict(K=-1.0), dict(K=0.0), dict(T=0.0), dict(F=float("inf")), dict(r=float("nan"))]
    for b in bad:
        args = dict(F=F, K=K, T=T, r=0.0)
        args.update(b)
        sig, st = orc.iv(0, 5.0, args["F"], args["K"], args["T"], args["r"], None, 1)
        assert st[0] == orc.INVALID and math.isnan(sig[0])


# ---------------------------------------------------------------------------
# conditioning (normalised vega, kappa) and the status margin: the quantities
# the parity tests use to gate and to excuse quotes
# ---------------------------------------------------------------------------
def _textbook_price_mp(model, SF, K, T, r, q, sigma, theta):
    """theta e^{-rT} [F Phi(theta d1) - K Phi(theta d2)] at mpmath's working
    precision (the caller sets it)."""
    SF, K, T, r, q = (mp.mpf(v) for v in (SF, K, T, r, q))
    F = SF if model == orc.BLACK76 else SF * mp.exp((r - q) * T)
    s = sigma * mp.sqrt(T)
    d1 = (mp.log(F / K) + s * s / 2) / s
    d2 = d1 - s
    return mp.exp(-r * T) * theta * (F * mp.ncdf(theta * d1) - K * mp.ncdf(theta * d2))


COND_CASES = [  # (model, S|F, K, T, r, q, sigma, flag): out of and in the money, wings, spot + dividends
    (orc.BLACK76, 100.0, 95.0, 0.25, 0.05, 0.0, 0.2, 1),
    (orc.BLACK76, 100.0, 95.0, 0.25, 0.05, 0.0, 0.2, -1),
    (orc.BLACK76, 100.0, 60.0, 2.0, 0.03, 0.0, 0.15, 1),
    (orc.BLACK76, 100.0, 160.0, 0.5, 0.01, 0.0, 0.9, 1),
    (orc.BLACK76, 100.0, 100.0, 1.0, 0.0, 0.0, 2.5, -1),
    (orc.BLACK76, 100.0, 140.0, 0.1, 0.02, 0.0, 0.4, -1),
    (orc.BSM, 100.0, 80.0, 1.5, 0.04, 0.02, 0.3, 1),
    (orc.BSM, 100.0, 125.0, 0.75, 0.02, 0.04, 0.6, -1),
    (orc.BSM, 100.0, 101.0, 3.0, 0.05, 0.01, 0.05, 1),
    (orc.BSM, 100.0, 30.0, 5.0, 0.06, 0.0, 1.2, -1),
]


def test_normalised_vega_is_the_price_derivative():
    # b'(x, s) = dP/dsigma / (e^{-rT} sqrt(F K) sqrt(T)): the derivative of the
    # textbook price by mpmath's numerical differentiation, in 50 digits
    for model, SF, K, T, r, q, sig, th in COND_CASES:
        v, _ = orc.conditioning(model, 1.0, SF, K, T, r, q, th, sig)
        with mp.workdps(50):
            vega = mp.diff(lambda x: _textbook_price_mp(model, SF, K, T, r, q, x, th), mp.mpf(sig))
            F = mp.mpf(SF) if model == orc.BLACK76 else SF * mp.exp((mp.mpf(r) - q) * T)
            want = vega / (mp.exp(-mp.mpf(r) * T) * mp.sqrt(F * K) * mp.sqrt(T))
        assert v[0] == pytest.approx(float(want), rel=1e-12), (model, SF, K, T, sig, th)


def test_kappa_is_the_sensitivity_of_sigma_to_the_price():
    # kappa = beta / (s b') = d ln(sigma) / d ln(P) (beta is proportional to P):
    # central differences of the definition's root at P (1 +- d), Richardson-
    # extrapolated from d and d/2, with d = 1e-6 / max(1, coarse estimate)
    # (the truncation error grows like d^2 kappa^3)
    def central(model, P, SF, K, T, r, q, th, d):
        Pp, Pm = P * (1 + d), P * (1 - d)
        sp, _ = orc.iv(model, Pp, SF, K, T, r, q, th)
        sm, _ = orc.iv(model, Pm, SF, K, T, r, q, th)
        mp.mp.dps = 30
        return mp.log(mp.mpf(sp[0]) / mp.mpf(sm[0])) / mp.log(mp.mpf(Pp) / mp.mpf(Pm))

    for model, SF, K, T, r, q, sig, th in COND_CASES:
        P = orc.price(model, SF, K, T, r, q, sig, th)[0]
        s0, st = orc.iv(model, P, SF, K, T, r, q, th)
        assert st[0] == orc.OK
        _, kap = orc.conditioning(model, P, SF, K, T, r, q, th, s0[0])
        d = 1e-6 / max(1.0, float(central(model, P, SF, K, T, r, q, th, 1e-6)))
        fd = (4 * central(model, P, SF, K, T, r, q, th, d / 2) -
              central(model, P, SF, K, T, r, q, th, d)) / 3
        assert kap[0] == pytest.approx(float(fd), rel=1e-6), (model, SF, K, T, sig, th)
    # in the money the intrinsic value dominates beta: kappa is large
    P = orc.price(orc.BLACK76, 100.0, 60.0, 1.0, 0.0, 0.0, 0.1, 1)[0]
    s0, _ = orc.iv(orc.BLACK76, P, 100.0, 60.0, 1.0, 0.0, None, 1)
    _, kap = orc.conditioning(orc.BLACK76, P, 100.0, 60.0, 1.0, 0.0, None, 1, s0[0])
    assert kap[0] > 1e3


def test_status_margin_counts_ulps_to_the_nearest_threshold():
    # Black-76 with r = 0 (no discounting), T = 1: beta = P / sqrt(F K).  Each
    # quote is built in 50 digits at k units of 2^-52 (relative) from one
    # threshold of the rule: below intrinsic at iota (1 - e_s), at intrinsic
    # at iota (1 + e_s), above the bound at b_max (1 - e_s) for the reduced
    # quote, with e_s = 64 * 2^-52.  The margin counts those units (relative
    # to beta for the in-the-money bound), up to the FP64 rounding of beta and
    # of the intrinsic value and bound (a few units).
    mp.mp.dps = 50
    F, u, es = 100.0, mp.mpf(2) ** -52, 64 * mp.mpf(2) ** -52
    cases = []
    for k in (-48, -20, -6, 6, 20, 48):
        for K, fl, which in ((90.0, 1, "below"), (110.0, -1, "below"), (90.0, 1, "at"),
                             (110.0, 1, "above"), (90.0, -1, "above"), (90.0, 1, "above")):
            cases.append((K, fl, which, k))
    for K, fl, which, k in cases:
        x = mp.log(mp.mpf(F) / K)
        itm = fl * x > 0
        iota = 2 * mp.sinh(abs(x) / 2) if itm else mp.mpf(0)
        bmax = mp.exp(-abs(x) / 2)
        if which == "below":
            beta, scale = iota * (1 - es) * (1 + k * u), 1
        elif which == "at":
            beta, scale = iota * (1 + es) * (1 + k * u), 1
        else:
            beta = iota + bmax * (1 - es) * (1 + k * u)
            scale = bmax / beta if beta > bmax else 1
        P = float(beta * mp.sqrt(mp.mpf(F) * K))
        if which != "above" and not itm:
            continue
        margin = orc.status(orc.BLACK76, P, F, K, 1.0, 0.0, None, fl)[3][0]
        want = float(abs(k) * scale)
        assert abs(margin - want) <= 2.0, (K, fl, which, k, margin, want)
        # and the decision on each side of the threshold, from the rule's
        # definition: below intrinsic under iota (1 - e_s); sigma = 0 up to
        # iota (1 + e_s); above the bound from b_max (1 - e_s) of the reduced quote
        sig, st = orc.iv(orc.BLACK76, P, F, K, 1.0, 0.0, None, fl)
        if which == "below":
            assert st[0] == (orc.BELOW_INTRINSIC if k < 0 else orc.OK), (K, fl, which, k)
            if k > 0:
                assert sig[0] == 0.0
        elif which == "at":
            assert st[0] == orc.OK and ((sig[0] == 0.0) if k < 0 else (sig[0] > 0.0)), (K, fl, which, k)
        else:
            assert st[0] == (orc.ABOVE_MAX if k > 0 else orc.OK), (K, fl, which, k)
            if k < 0:
                assert sig[0] > 0.0
    # far from every threshold the margin is large; an invalid quote has none
    assert orc.status(orc.BLACK76, 12.0, F, 90.0, 1.0, 0.0, None, 1)[3][0] > 1e10
    assert orc.status(orc.BLACK76, 5.0, F, 90.0, 1.0, 0.0, None, 0)[3][0] == np.inf


def test_paper_quick_use_example():
    with open(os.path.join(GOLDEN, "paper_quick_use.json")) as f:
        g = json.load(f)
    K = np.array(g["K"])
    n = K.size
    flag = np.array([1 if c == "c" else -1 for c in g["flag"]], np.int8)
    S, t, r = np.full(n, g["S"]), np.full(n, g["t"]), np.full(n, g["r"])
    P = orc.price(orc.BLACK_SCHOLES, S, K, t, r, None, np.full(n, g["sigma"]), flag)
    sig, st = orc.iv(orc.BLACK_SCHOLES, P, S, K, t, r, None, flag)
    assert np.all(st == orc.OK)
    np.testing.assert_allclose(sig, g["expected_iv"], rtol=1e-14)


# ---------------------------------------------------------------------------
# the step-by-step solvers of Section 2.2 against the definition
# ---------------------------------------------------------------------------
def _grid():
    xs = -np.concatenate([[0.0], np.logspace(-8, np.log10(8.0), 40)])
    ss = np.logspace(-3, np.log10(12.0), 60)
    X, S = np.meshgrid(xs, ss, indexing="ij")
    X, S = X.ravel(), S.ravel()
    n = X.size
    w = dict(model=0, S_or_F=np.ones(n), K=np.exp(-X), T=np.ones(n), r=np.zeros(n), q=None,
             flag=np.ones(n, np.int8), sigma_true=S)
    return wl.fill_prices(w, orc.price)


@pytest.fixture(scope="module")
def grid_truth():
    w = _grid()
    sig, st = orc.iv(0, w["P"], w["S_or_F"], w["K"], w["T"], w["r"], None, w["flag"])
    v, kap = _gate(0, w["P"], w, sig)
    solved = (st == orc.OK) & (sig > 0) & (w["P"] > 1e-300)
    return w, sig, st, v, kap, solved


@pytest.mark.parametrize("n_iter", [2, 3])
def test_lbr_reaches_machine_precision_in_two_iterations(grid_truth, n_iter):
    w, sig, st, v, kap, solved = grid_truth
    sl, st2, reg = orc.iv_lbr(0, w["P"], w["S_or_F"], w["K"], w["T"], w["r"], None, w["flag"],
                              n_iter=n_iter)
    assert np.array_equal(st, st2)
    # all four initial-guess regions are exercised
    assert set(np.unique(reg[solved])) == {0, 1, 2, 3}
    rel = np.abs(sl[solved] - sig[solved]) / sig[solved]
    assert np.all(rel <= 4 * EPS * (1 + kap[solved]))
    gate = (v[solved] > 1e-8) & (kap[solved] <= 1e3)
    assert rel[gate].max() <= 1e-12


def test_fp64_normalised_black_against_binary128():
    # the oracle's own FP64 evaluation (erfcx difference with a continued-
    # fraction erfcx, small-t Mills-ratio series, CDF-direct past the
    # inflection point) against the binary128 definition
    xs = np.concatenate([-np.logspace(-8, np.log10(40), 60), [0.0], np.logspace(-8, np.log10(40), 60)])
    ss = np.logspace(-4, np.log10(50), 90)
    X, S = np.meshgrid(xs, ss, indexing="ij")
    X, S = X.ravel(), S.ravel()
    for th in (1, -1):
        ref = orc.normalised_black(X, S, th)
        got = orc.normalised_black_f64(X, S, th)
        m = ref > 1e-300
        rel = np.abs(got[m] - ref[m]) / ref[m]
        h = np.abs(X[m]) / S[m]
        # |h| <= 10: the series and the erfcx difference both keep 13 digits
        # (a few hundred ulp at most, the recurrence's and the exponent's loss)
        assert rel[h <= 10].max() <= 1e-13, rel[h <= 10].max()
        # beyond, the erfcx difference loses log10(|h|/2t) digits for small t
        assert rel.max() <= 2e-10, rel.max()
    # at the money b = erf(s / (2 sqrt 2)) (series below t = 0.1, CDF-direct above)
    for s_ in (1e-4, 0.05, 0.199, 0.2, 1.0, 4.0, 20.0):
        got = orc.normalised_black_f64(0.0, s_, 1)[0]
        assert got == pytest.approx(float(mp.erf(mp.mpf(s_) / (2 * mp.sqrt(2)))), rel=2e-15), s_
    # the erfcx difference on both sides of the erfcx switch at z = 2: t = 1/2
    # and -(h + t)/sqrt2 = z, so the first erfcx argument crosses 2
    zs = np.array([1.5, 1.999999, 2.0, 2.000001, 2.5, 6.0, 30.0])
    h = -np.sqrt(2.0) * zs - 0.5
    x, s_ = 2.0 * h * 0.5, np.full(zs.size, 1.0)
    ref = orc.normalised_black(x, s_, 1)
    got = orc.normalised_black_f64(x, s_, 1)
    m = ref > 1e-300
    assert np.all(np.abs(got[m] - ref[m]) <= 1e-13 * ref[m])


def test_fp64_lbr_against_the_definition(grid_truth):
    # the FP64 CPU solver (the benchmark's CPU baseline): the LBR steps with
    # the FP64 normalised Black reach the definition within 16 eps (1 + kappa)
    w, sig, st, v, kap, solved = grid_truth
    sl, st2, reg = orc.iv_lbr_f64(0, w["P"], w["S_or_F"], w["K"], w["T"], w["r"], None, w["flag"],
                                  n_iter=3)
    assert np.array_equal(st, st2)
    assert set(np.unique(reg[solved])) == {0, 1, 2, 3}
    rel = np.abs(sl[solved] - sig[solved]) / sig[solved]
    gate = (v[solved] > 1e-8) & (kap[solved] <= 1e3)
    assert rel[gate].max() <= 1e-12
    assert np.all(rel[v[solved] > 1e-8] <= 16 * EPS * (1 + kap[solved][v[solved] > 1e-8]))


def test_lbr_one_iteration_is_not_enough(grid_truth):
    w, sig, st, v, kap, solved = grid_truth
    sl, _, _ = orc.iv_lbr(0, w["P"], w["S_or_F"], w["K"], w["T"], w["r"], None, w["flag"], n_iter=1)
    rel = np.abs(sl[solved] - sig[solved]) / sig[solved]
    assert rel.max() > 1e-9


def test_halley_with_bisection_fallback(grid_truth):
    w, sig, st, v, kap, solved = grid_truth
    sh, st2, fb = orc.iv_halley(0, w["P"], w["S_or_F"], w["K"], w["T"], w["r"], None, w["flag"])
    assert np.array_equal(st, st2)
    rel = np.abs(sh[solved] - sig[solved]) / sig[solved]
    assert np.all(rel <= 8 * EPS * (1 + kap[solved]))
    # near the money the eight Halley sweeps converge without the fallback
    atm = solved & (np.abs(np.log(w["K"])) < 0.05) & (w["sigma_true"] > 0.05) & (w["sigma_true"] < 2)
    assert fb[atm].mean() < 0.05


def test_halley_sweeps_failure_share():
    # How often the method itself needs the fallback (Section 2.2: "typically
    # < 0.5 %" on the paper's grid and tolerance): the oracle's eight plain
    # sweeps from the Brenner-Subrahmanyam start, no early exit, tested at a
    # relative Newton distance of 1e-10.  Near the money they converge; on
    # Black-76 quotes of the small configuration's distribution (short
    # maturities, |ln K/F| up to 1/2) about three in ten do not, and on a slice
    # of the benchmark grid (log-moneyness to +-3) most do not.
    w = wl.fill_prices(wl.black76_quotes(100000, seed=5), orc.price_f64)
    _, st, fb = orc.iv_halley(0, w["P"], w["S_or_F"], w["K"], w["T"], w["r"], None, w["flag"])
    share = fb[st == orc.OK].astype(bool).mean()
    assert 0.2 < share < 0.4, share
    near = (st == orc.OK) & (np.abs(np.log(w["K"] / w["S_or_F"])) < 0.05) & (w["T"] > 0.25)
    assert fb[near].astype(bool).mean() < 0.01
    g = wl.fill_prices(wl.bsm_grid(4096, 64, seed=1), orc.price_f64)
    _, st, fb = orc.iv_halley(2, g["P"], g["S_or_F"], g["K"], g["T"], g["r"], g["q"], g["flag"])
    assert 0.6 < fb[st == orc.OK].astype(bool).mean() < 0.85


def test_solvers_on_in_the_money_quotes():
    w = wl.fill_prices(wl.black76_quotes(1024, seed=21), orc.price)
    sig, st = orc.iv(0, w["P"], w["S_or_F"], w["K"], w["T"], w["r"], None, w["flag"])
    v, kap = _gate(0, w["P"], w, sig)
    ok = (st == 0) & (sig > 0)
    for fn in (lambda: orc.iv_lbr(0, w["P"], w["S_or_F"], w["K"], w["T"], w["r"], None, w["flag"]),
               lambda: orc.iv_halley(0, w["P"], w["S_or_F"], w["K"], w["T"], w["r"], None, w["flag"])):
        s2, st2, _ = fn()
        assert np.array_equal(st, st2)
        rel = np.abs(s2[ok] - sig[ok]) / sig[ok]
        assert np.all(rel <= 8 * EPS * (1 + kap[ok]))


@pytest.mark.parametrize("model", [orc.BLACK_SCHOLES, orc.BSM])
def test_solvers_on_spot_quotes_with_dividends(model):
    # the FP64 normalisation x = ln(S/K) + (r - q) T feeds both solvers
    w = wl.fill_prices(wl.bsm_quotes(1024, seed=22), orc.price)
    if model == orc.BLACK_SCHOLES:
        w = dict(w, model=model, q=None)
        wl.fill_prices(w, orc.price)
    sig, st = orc.iv(model, w["P"], w["S_or_F"], w["K"], w["T"], w["r"], w["q"], w["flag"])
    v, kap = _gate(model, w["P"], w, sig)
    ok = (st == 0) & (sig > 0)
    assert ok.mean() > 0.9
    for fn in (orc.iv_lbr, orc.iv_halley):
        s2, st2, _ = fn(model, w["P"], w["S_or_F"], w["K"], w["T"], w["r"], w["q"], w["flag"])
        assert np.array_equal(st, st2)
        rel = np.abs(s2[ok] - sig[ok]) / sig[ok]
        assert np.all(rel <= 8 * EPS * (1 + kap[ok]))


def test_lbr_interior_guess_is_a_hermite_interpolant():
    # Section 2.2: the interior guess interpolates s(beta) between the
    # boundary points s_l < s_c < s_h (inflection s_c = sqrt(2|x|), tangent
    # feet s_l, s_h) with the slopes ds/dbeta = 1/b' there.  The guess is the
    # LBR's output after zero iterations.
    for x in (-0.05, -0.5, -2.0):
        bmax = math.exp(0.5 * x)
        vega = lambda s: math.exp(-0.5 * ((x / s) ** 2 + (0.5 * s) ** 2)) / math.sqrt(2 * math.pi)
        b = lambda s: float(orc.normalised_black(np.array([x]), np.array([s]), 1)[0])
        sc = math.sqrt(-2 * x)
        bc, vc = b(sc), vega(sc)
        sl, sh = sc - bc / vc, sc + (bmax - bc) / vc
        bl, vl, bh, vh = b(sl), vega(sl), b(sh), vega(sh)
        # quotes at beta = end + k delta, k = 1, 2 (F = 1, K = e^{-x}, T = 1, r = 0)
        for b0, s0, v0, b1, sign in ((bl, sl, vl, bc, 1), (bc, sc, vc, bl, -1),
                                     (bc, sc, vc, bh, 1), (bh, sh, vh, bc, -1)):
            d = 1e-6 * abs(b1 - b0) * sign
            beta = np.array([b0 + d, b0 + 2 * d])
            K = np.full(2, math.exp(-x))
            P = beta * np.sqrt(K)
            g, st, _ = orc.iv_lbr(0, P, np.ones(2), K, np.ones(2), np.zeros(2), None,
                                  np.ones(2, np.int8), n_iter=0)
            assert np.all(st == orc.OK)
            assert g[0] == pytest.approx(s0 + d / v0, rel=1e-6, abs=1e-9)
            assert (g[1] - g[0]) / d == pytest.approx(1 / v0, rel=1e-3)


# ---------------------------------------------------------------------------
# Greeks and the implicit-function gradient
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("model", [orc.BLACK76, orc.BLACK_SCHOLES, orc.BSM])
def test_greeks_against_finite_differences(model):
    w = wl.bsm_quotes(64, seed=7)
    S, K, T, r, q, sg, fl = (w[k] for k in ("S_or_F", "K", "T", "r", "q", "sigma_true", "flag"))
    qq = q if model == orc.BSM else None
    d, g, vg, th, rho = orc.greeks(model, S, K, T, r, qq, sg, fl)
    P = lambda S_=S, K_=K, T_=T, r_=r, s_=sg: orc.price(model, S_, K_, T_, r_, qq, s_, fl)

    # fourth-order central stencils
    def d1(f, h):
        return (-f(2 * h) + 8 * f(h) - 8 * f(-h) + f(-2 * h)) / (12 * h)

    def d2(f, h):
        return (-f(2 * h) + 16 * f(h) - 30 * f(0 * h) + 16 * f(-h) - f(-2 * h)) / (12 * h * h)

    hS = 1e-3 * S
    fd_d = d1(lambda e: P(S_=S + e), hS)
    fd_g = d2(lambda e: P(S_=S + e), hS)
    fd_v = d1(lambda e: P(s_=sg + e), 1e-4 * sg) * 0.01
    fd_t = -d1(lambda e: P(T_=T + e), 1e-4 * T) / 365
    fd_r = d1(lambda e: P(r_=r + e), np.full_like(r, 1e-4)) * 0.01
    np.testing.assert_allclose(d, fd_d, rtol=1e-8, atol=1e-11)
    np.testing.assert_allclose(g, fd_g, rtol=1e-6, atol=1e-10)
    np.testing.assert_allclose(vg, fd_v, rtol=1e-8, atol=1e-11)
    np.testing.assert_allclose(th, fd_t, rtol=1e-8, atol=1e-11)
    np.testing.assert_allclose(rho, fd_r, rtol=1e-8, atol=1e-11)


def test_greeks_textbook_values():
    # S = K = 100, T = 1, r = 5%, sigma = 20%: d1 = 0.35, delta = N(0.35)
    d, g, vg, th, rho = orc.greeks(orc.BLACK_SCHOLES, 100.0, 100.0, 1.0, 0.05, None, 0.2, 1)
    assert d[0] == pytest.approx(0.5 * math.erfc(-0.35 / math.sqrt(2)), rel=1e-15)
    assert g[0] == pytest.approx(math.exp(-0.35 ** 2 / 2) / math.sqrt(2 * math.pi) / 20.0, rel=1e-15)


@pytest.mark.parametrize("model", [orc.BLACK76, orc.BSM])
def test_iv_gradient_against_finite_differences(model):
    w = wl.bsm_quotes(48, seed=8)
    if model == orc.BLACK76:
        w["q"] = None
    w = wl.fill_prices(w, orc.price)
    args = [w[k] for k in ("S_or_F", "K", "T", "r")]
    q = w["q"]
    sig, st = orc.iv(model, w["P"], *args, q, w["flag"])
    ok = (st == 0) & (sig > 0)
    gs = np.ones(sig.size)
    grads = orc.iv_grad(model, *args, q, w["flag"], sig, st, gs)

    def iv_at(**kw):
        a = dict(P=w["P"], S=args[0], K=args[1], T=args[2], r=args[3], q=q)
        a.update(kw)
        return orc.iv(model, a["P"], a["S"], a["K"], a["T"], a["r"], a["q"], w["flag"])[0]

    rel_h = 1e-6
    names = ["P", "S", "K", "T", "r"] + (["q"] if model == orc.BSM else [])
    base = dict(P=w["P"], S=args[0], K=args[1], T=args[2], r=args[3], q=q)
    for k, name in enumerate(names):
        x0 = base[name]
        h = rel_h * np.abs(x0) if name in ("P", "S", "K", "T") else np.full(sig.size, 1e-6)
        fd = (iv_at(**{name: x0 + h}) - iv_at(**{name: x0 - h})) / (2 * h)
        np.testing.assert_allclose(grads[k][ok], fd[ok], rtol=2e-6, atol=1e-8, err_msg=name)
    if model != orc.BSM:
        assert np.all(grads[5] == 0)
