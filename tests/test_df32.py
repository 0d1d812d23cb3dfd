"""The kernels' double-float functions, built for the host and checked on the CPU.

The mixed solver's Householder(3) correction (Section 2.2: FP32 iterations,
then one step at FP64 accuracy) evaluates its normalised Black residual in
double-float arithmetic (csrc/fv_df32.cuh, tables from csrc/gen_df32_tables.py):
pairs of FP32 numbers carrying ~48 bits.  The header compiles as plain C++;
here it is built with the host compiler (no contraction, exactly rounded FMA,
the same operations as on the device) and every function is compared with
mpmath on points spread over its range, and the correction itself with the
exact root of the normalised Black equation.
"""
import ctypes
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")
mp.mp.dps = 50

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2604_27210_gb300", "csrc")
HARNESS = os.path.join(ROOT, "tests", "df32_harness.cpp")
EPS48 = 2.0 ** -48


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    out = str(tmp_path_factory.mktemp("df32") / "libdf32h.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-I", CSRC,
                    HARNESS, "-o", out], check=True)
    L = ctypes.CDLL(out)
    f, d, i = ctypes.c_float, ctypes.c_double, ctypes.c_int
    fp = ctypes.POINTER(ctypes.c_float)
    L.h_dexp.argtypes = [f, f, fp]
    L.h_dlog.argtypes = [f, f, fp]
    L.h_dlog_of.argtypes = [d, fp]
    L.h_derfcx.argtypes = [f, f, fp]
    L.h_df_of.argtypes = [d, fp]
    L.h_df_of.restype = i
    L.h_drsqrt.argtypes = [f, f, fp]
    L.h_nb.argtypes = [d, f, i, fp]
    L.h_nb.restype = i
    L.h_corr.argtypes = [d, d, d, d, d, f, i, ctypes.POINTER(ctypes.c_double)]
    L.h_corr.restype = i
    L.h_dlog1p.argtypes = [f, f, fp]
    L.h_dexp_em1.argtypes = [f, f, fp]
    vp = ctypes.c_void_p
    L.h_decide.argtypes = [i, vp, vp, vp, vp, vp, vp, vp, ctypes.c_long, vp, vp]
    return L


def f32(v):
    return struct.unpack("<f", struct.pack("<f", float(v)))[0]


def split(v):
    """A double-float pair for the mpmath number v."""
    hi = f32(v)
    return hi, f32(mp.mpf(v) - hi)


def val(pair):
    return mp.mpf(float(pair[0])) + mp.mpf(float(pair[1]))


def call2(fn, *args):
    out = (ctypes.c_float * 8)()
    r = fn(*args, out)
    return r, (out[0], out[1])


def test_df_of_and_widening(lib):
    g = np.random.default_rng(1)
    for d in np.concatenate([g.uniform(-1e3, 1e3, 200), 10.0 ** g.uniform(-29, 37, 200),
                             [1.0, -2.5, 1e-30, 3e37]]):
        ok, p = call2(lib.h_df_of, float(d))
        assert ok == 1
        assert abs(float(val(p) - mp.mpf(float(d)))) <= 2.0 ** -47 * abs(d)
        # head and tail do not overlap
        assert abs(p[1]) <= abs(p[0]) * 2.0 ** -23
    for d in (0.0, 1e-31, 1e39, float("inf"), float("nan")):
        assert call2(lib.h_df_of, d)[0] == 0


def test_exp_within_2_46(lib):
    g = np.random.default_rng(2)
    worst = 0.0
    for a in np.concatenate([g.uniform(-70, 87, 3000), g.uniform(-0.01, 0.01, 300), [0.0]]):
        ah, al = split(mp.mpf(float(a)) + mp.mpf(g.uniform(-1, 1)) * 1e-9 * abs(float(a)))
        _, r = call2(lib.h_dexp, ah, al)
        ref = mp.exp(val((ah, al)))
        worst = max(worst, abs(float((val(r) - ref) / ref)))
    assert worst <= 2.0 ** -46, worst


def test_exp_and_expm1_from_one_reduction(lib):
    g = np.random.default_rng(12)
    we, wm = 0.0, 0.0
    for a in np.concatenate([-10.0 ** g.uniform(-9, 1.8, 3000), [0.0, -0.005, -0.00499, -0.0051]]):
        ah, al = split(mp.mpf(float(a)))
        out = (ctypes.c_float * 4)()
        lib.h_dexp_em1(ah, al, out)
        aa = val((ah, al))
        we = max(we, abs(float((val((out[0], out[1])) - mp.exp(aa)) / mp.exp(aa))))
        if aa != 0:
            wm = max(wm, abs(float((val((out[2], out[3])) - mp.expm1(aa)) / mp.expm1(aa))))
    # expm1 to 2^-44: the table holds 2^(j/128) to 2^-48, the result is down to
    # ~1/80 of it just above the unreduced range |a| < 1/200
    assert we <= 2.0 ** -46 and wm <= 2.0 ** -44, (we, wm)


def test_log_within_2_46(lib):
    # relative to max(1, |ln y|): a double-float holds ~2^-48 of its value,
    # and the sum m ln2 + L_j + log1p(r) rounds three times
    g = np.random.default_rng(3)
    worst = 0.0
    ys = np.concatenate([10.0 ** g.uniform(-37, 37, 3000), 1.0 + g.uniform(-0.02, 0.02, 500)])
    for y in ys:
        yh, yl = split(mp.mpf(float(y)) * (1 + mp.mpf(g.uniform(-1, 1)) * 1e-8))
        _, r = call2(lib.h_dlog, yh, yl)
        ref = mp.log(val((yh, yl)))
        worst = max(worst, abs(float(val(r) - ref)) / max(1.0, abs(float(ref))))
    assert worst <= 2.0 ** -46, worst


def test_log_of_double_over_the_fp64_range(lib):
    g = np.random.default_rng(4)
    worst = 0.0
    for y in np.concatenate([10.0 ** g.uniform(-307, 308, 3000), 1.0 + g.uniform(-0.3, 0.4, 500)]):
        _, r = call2(lib.h_dlog_of, float(y))
        ref = mp.log(mp.mpf(float(y)))
        worst = max(worst, abs(float(val(r) - ref)) / max(1.0, abs(float(ref))))
    assert worst <= 2.0 ** -46, worst


def erfcx(z):
    return mp.exp(z * z) * mp.erfc(z)


def test_erfcx_within_2_46_on_every_piece_and_the_asymptote(lib):
    g = np.random.default_rng(5)
    zs = [0.0, 1e-6, 0.03125, 0.5, 0.49999997, 1.0, 127.99999, 128.0, 1e3, 1e6, 1e15]
    # every piece: 8 uniform below 1/2, 16 per binade up to 128
    edges = [k / 16 for k in range(9)] + [2.0 ** e * (1 + j / 16) for e in range(-1, 7)
                                          for j in range(1, 17)]
    for a, b in zip(edges[:-1], edges[1:]):
        zs += list(g.uniform(a, b, 12)) + [a, np.nextafter(np.float32(b), np.float32(0))]
    worst = 0.0
    for z in zs:
        zh, zl = split(mp.mpf(float(z)) * (1 + mp.mpf(g.uniform(-1, 1)) * 1e-8))
        if zh < 0:
            continue
        _, r = call2(lib.h_derfcx, zh, zl)
        zz = val((zh, zl))
        ref = erfcx(zz)
        worst = max(worst, abs(float((val(r) - ref) / ref)))
    assert worst <= 2.0 ** -46, worst


def test_rsqrt_within_2_46(lib):
    g = np.random.default_rng(6)
    worst = 0.0
    for y in 10.0 ** g.uniform(-29, 29, 500):
        yh, yl = split(mp.mpf(float(y)))
        _, r = call2(lib.h_drsqrt, yh, yl)
        ref = 1 / mp.sqrt(val((yh, yl)))
        worst = max(worst, abs(float((val(r) - ref) / ref)))
    assert worst <= 2.0 ** -46, worst


# ---------------------------------------------------------------------------
# the normalised Black evaluation and the correction step
# ---------------------------------------------------------------------------
def nb(x, s):
    """b(x, s) of the call, x <= 0, in mpmath."""
    x, s = mp.mpf(x), mp.mpf(s)
    return mp.exp(x / 2) * mp.ncdf(x / s + s / 2) - mp.exp(-x / 2) * mp.ncdf(x / s - s / 2)


def nb_prime(x, s):
    x, s = mp.mpf(x), mp.mpf(s)
    return mp.npdf(x / s + s / 2) * mp.exp(x / 2)


def region(x, beta):
    """The LBR region of the reduced quote (x <= 0, 0 < beta < e^{x/2}),
    from the boundaries of Section 2.2 evaluated in mpmath."""
    x = mp.mpf(x)
    bmax = mp.exp(x / 2)
    if x == 0:
        return 1 if beta <= nb(x, mp.mpf(2)) else 2
    sc = mp.sqrt(-2 * x)
    bc = nb(x, sc)
    vc = nb_prime(x, sc)
    sl = sc - bc / vc
    sh = sc + (bmax - bc) / vc
    if beta <= bc:
        if sl <= 0:
            return 1
        return 0 if beta < nb(x, sl) else 1
    return 2 if beta <= nb(x, sh) else 3


def b_over_e(x, s):
    h, t = mp.mpf(x) / s, mp.mpf(s) / 2
    return nb(x, s) / mp.exp(-(h * h + t * t) / 2)


# (x, s) over the LBR's regions and the evaluation's branches: near the money
# and deep out of it, small t (series) and large t, past the inflection point
CASES = [(-0.01, 0.005), (-0.01, 0.05), (-0.01, 0.15), (-0.01, 3.0), (-0.2, 0.05), (-0.2, 0.15),
         (-0.2, 0.6), (-0.2, 2.0), (-0.5, 0.02), (-0.5, 0.12), (-0.5, 0.5), (-0.5, 1.0),
         (-0.5, 5.0), (-1.5, 0.05), (-1.5, 0.3), (-1.5, 1.7), (-1.5, 4.0), (-3.0, 0.1),
         (-3.0, 0.5), (-3.0, 2.4), (-3.0, 6.0), (-8.0, 0.4), (-8.0, 3.0), (-8.0, 9.0),
         (0.0, 0.01), (0.0, 0.3), (0.0, 2.0), (-0.7, 0.04), (-0.9, 0.03), (-30.0, 1.0),
         (-30.0, 7.7), (-30.0, 12.0), (-0.001, 0.0002), (-0.001, 0.0006)]


@pytest.mark.parametrize("x,s", CASES)
def test_normalised_black_value_or_complement(lib, x, s):
    beta = nb(x, s)
    reg = region(x, beta)
    s32 = f32(s)
    out = (ctypes.c_float * 8)()
    assert lib.h_nb(float(x), s32, reg, out) == 1
    B = val((out[0], out[1]))
    E = val((out[2], out[3]))
    h, t = mp.mpf(float(x)) / mp.mpf(s32), mp.mpf(s32) / 2
    assert abs(float((E - (h * h + t * t) / 2) / E if E else E)) <= 2.0 ** -46
    via_comp = out[6] == 1.0
    b = nb(float(x), s32)
    e = mp.exp(-(h * h + t * t) / 2)
    ref = (mp.exp(mp.mpf(float(x)) / 2) - b) / e if (reg == 3 or via_comp) else b / e
    rel = abs(float((B - ref) / ref))
    if reg == 0:
        # log space: B's error only moves ln b, by rel, and s by rel/h^2
        assert rel <= 2.0 ** -44 * max(1.0, float(h * h)), rel
    else:
        assert rel <= 2.0 ** -44, rel


def root(x, beta, s0):
    """The exact root s of b(x, s) = beta (mpmath, from s0)."""
    return mp.findroot(lambda s: nb(x, s) - beta, mp.mpf(s0), tol=mp.mpf(10) ** -40)


@pytest.mark.parametrize("x,s", CASES)
def test_correction_from_an_fp32_iterate_reaches_the_root(lib, x, s):
    # the reduced quote as FP64 numbers, the FP32 iterate 3e-7 off the root
    g = np.random.default_rng(int(abs(x) * 1000 + s * 100))
    beta = float(nb(x, s))
    bmax = float(mp.exp(mp.mpf(x) / 2))
    c_beta = float(mp.exp(mp.mpf(x) / 2) - mp.mpf(beta))
    reg = region(x, mp.mpf(beta))
    T = float(g.uniform(0.1, 3.0))
    s_true = root(mp.mpf(x), mp.mpf(beta), s)
    sigma_true = s_true / mp.sqrt(mp.mpf(T))
    # the residual is evaluated to ~2^-46 relative in the quantity it is formed
    # from: b itself, or b_max - b for the highest region and past the
    # inflection point; its error moves s by that quantity / (s b') times it
    b = nb(x, s_true)
    past = reg == 3 or (reg in (1, 2) and mp.mpf(x) / s_true + s_true / 2 > 0)
    cond = float((mp.exp(mp.mpf(x) / 2) - b if past else b) / (s_true * nb_prime(x, s_true)))
    for delta in (3e-7, -2e-7, 1e-5):
        s32 = f32(s_true * (1 + delta))
        sig = ctypes.c_double(0.0)
        ok = lib.h_corr(beta, c_beta, float(x), 0.0, T, s32, reg, ctypes.byref(sig))
        assert ok == 1, (x, s, reg)
        rel = abs(float((mp.mpf(sig.value) - sigma_true) / sigma_true))
        assert rel <= 2.0 ** -44 * (1 + cond), (x, s, reg, delta, rel, cond)
    assert bmax > beta


def test_correction_declines_outside_its_range(lib):
    sig = ctypes.c_double(0.0)
    # beta below the double-float range in a middle region
    assert lib.h_corr(1e-40, 0.5, -0.01, 0.0, 1.0, f32(0.001), 1, ctypes.byref(sig)) == 0
    # e^E beyond the range of the middle regions' direct form
    assert lib.h_corr(1e-3, 0.5, -200.0, 0.0, 1.0, f32(1.0), 1, ctypes.byref(sig)) == 0
    # non-positive or non-finite iterate
    assert lib.h_corr(0.1, 0.5, -0.1, 0.0, 1.0, 0.0, 1, ctypes.byref(sig)) == 0
    assert lib.h_corr(0.1, 0.5, -0.1, 0.0, 1.0, float("inf"), 1, ctypes.byref(sig)) == 0


def test_committed_tables_are_the_generators_output(tmp_path):
    import importlib.util
    spec = importlib.util.spec_from_file_location("gen_df32_tables",
                                                  os.path.join(CSRC, "gen_df32_tables.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    out = gen.write(str(tmp_path / "fv_df32_tables.h"))
    assert open(out).read() == open(os.path.join(CSRC, "fv_df32_tables.h")).read()


def test_log1p_keeps_the_relative_precision_of_u(lib):
    g = np.random.default_rng(7)
    worst = 0.0
    us = np.concatenate([g.uniform(-0.5, 1.0, 2000), g.uniform(-1e-2, 1e-2, 500),
                         np.sign(g.uniform(-1, 1, 500)) * 10.0 ** g.uniform(-12, -3, 500),
                         [k / 128 for k in range(-64, 129)], [0.0]])
    for u in us:
        uh, ul = split(mp.mpf(float(u)) * (1 + mp.mpf(g.uniform(-1, 1)) * 1e-8))
        _, r = call2(lib.h_dlog1p, uh, ul)
        ref = mp.log1p(val((uh, ul)))
        if ref == 0:
            assert val(r) == 0
            continue
        worst = max(worst, abs(float((val(r) - ref) / ref)))
    # -ln c_j and log1p(r) may cancel by a factor ~2 half-way between rows
    assert worst <= 2.0 ** -45, worst


# ---------------------------------------------------------------------------
# the double-float status rule against the oracle's FP64 rule
# ---------------------------------------------------------------------------
def _decide(lib, w):
    n = len(w["P"])
    cols = [np.ascontiguousarray(np.asarray(w[k], dtype=np.float64)) for k in
            ("P", "S_or_F", "K", "T", "r")]
    q = np.ascontiguousarray(np.zeros(n) if w.get("q") is None else np.asarray(w["q"], np.float64))
    flag = np.ascontiguousarray(np.asarray(w["flag"], dtype=np.int8))
    out = np.empty((n, 4), np.int32)
    vals = np.empty((n, 10), np.float32)
    lib.h_decide(int(w["model"]), *[c.ctypes.data for c in cols], q.ctypes.data, flag.ctypes.data,
                 n, out.ctypes.data, vals.ctypes.data)
    v = vals.astype(np.float64)
    return out, {k: v[:, 2 * i] + v[:, 2 * i + 1] for i, k in
                 enumerate(("beta", "x", "bmax", "c_beta", "ln_beta"))}


def _workloads():
    from oracle import oracle as orc
    from paper_2604_27210_gb300 import workloads as wl
    out = []
    g = wl.fill_prices(wl.bsm_grid(512, 256, seed=1), orc.price)
    out.append(("bsm grid", g))
    out.append(("black76", wl.fill_prices(wl.black76_quotes(50000, seed=3), orc.price)))
    out.append(("bsm quotes", wl.fill_prices(wl.bsm_quotes(50000, seed=4), orc.price)))
    return out


@pytest.mark.parametrize("name", ["bsm grid", "black76", "bsm quotes"])
def test_status_rule_in_double_float_matches_the_fp64_rule(lib, name):
    from oracle import oracle as orc
    w = dict(_workloads())[name]
    n = len(w["P"])
    out, v = _decide(lib, w)
    st, x, beta, margin = orc.status(w["model"], *[w[k] for k in ("P", "S_or_F", "K", "T", "r",
                                                                     "q", "flag")])
    dec = out[:, 2] == 0
    # every quote the double-float rule decides has the FP64 rule's status
    assert np.array_equal(out[dec, 0], st[dec]), (out[dec, 0] != st[dec]).sum()
    # in the money the reduced price beta - iota is taken here only where it
    # keeps at least half of beta; out of the money most quotes are decided here
    itm = (np.asarray(w["flag"]) * x > 0) & (st != orc.INVALID)
    iota = np.where(itm, 2 * np.sinh(np.abs(x) / 2), 0.0)
    beta_otm = beta - iota
    assert np.all(beta_otm[dec & itm & (out[:, 1] == 1)] >= 0.49 * beta[dec & itm & (out[:, 1] == 1)])
    otm = ~itm & (st != orc.INVALID)
    assert dec[otm].mean() > 0.97, dec[otm].mean()
    if itm.sum() > 0.1 * n:
        assert dec[itm].mean() > 0.2, dec[itm].mean()
    # the reduced quote of the solved ones, against the FP64 rule's values
    solve = dec & (out[:, 1] == 1)
    assert solve.sum() > 0.3 * n
    norm = solve & (out[:, 3] == 0)
    rel_x = np.abs(-np.abs(x[norm]) - v["x"][norm]) / np.abs(x[norm])
    rel_b = np.abs(beta_otm[norm] - v["beta"][norm]) / beta_otm[norm]
    assert rel_x.max() <= 2.0 ** -42, rel_x.max()
    assert rel_b.max() <= 2.0 ** -42, rel_b.max()
    bmax = np.exp(-np.abs(x[norm]) / 2)
    assert np.all(np.abs(v["bmax"][norm] - bmax) <= 2.0 ** -44 * bmax)
    assert np.all(np.abs(v["c_beta"][norm] - (bmax - beta_otm[norm])) <= 2.0 ** -42 * bmax)
    tiny = solve & (out[:, 3] == 1)
    if tiny.any():
        assert np.all(np.abs(v["ln_beta"][tiny] - np.log(beta[tiny])) <= 2.0 ** -44 * np.abs(np.log(beta[tiny])))


def test_status_rule_in_double_float_edge_cases(lib):
    from oracle import oracle as orc
    F, K, T, r = 100.0, 120.0, 0.5, 0.03
    bmax_price = K * np.exp(-r * T)  # a put's bound: the discounted strike
    # call out of the money (F < K): bound F e^{-rT}; put in the money
    P = np.array([0.0, -0.0, -1e-3, 1e-310, 1e-200, 5.0, F * np.exp(-r * T) * (1 - 1e-15),
                  F * np.exp(-r * T) * (1 + 1e-12), F * np.exp(-r * T) * (1 - 1e-9), np.nan, 5.0,
                  5.0, 5.0])
    n = len(P)
    w = {"model": 0, "P": P, "S_or_F": np.array([F] * 10 + [np.inf, F, F]),
         "K": np.array([K] * 11 + [-1.0, K]), "T": np.full(n, T), "r": np.full(n, r), "q": None,
         "flag": np.array([1] * 12 + [2], np.int8)}
    out, v = _decide(lib, w)
    st, x, beta, margin = orc.status(0, w["P"], w["S_or_F"], w["K"], w["T"], w["r"], None, w["flag"])
    dec = out[:, 2] == 0
    assert np.array_equal(out[dec, 0], st[dec])
    assert list(out[:3, 0]) == [orc.OK, orc.OK, orc.BELOW_INTRINSIC] and list(out[:3, 1]) == [0, 0, 0]
    assert out[3, 2] == 1  # FP64 beta would be subnormal: the FP64 rule
    assert out[4, 3] == 1 and out[4, 1] == 1  # tiny price: carried as ln beta
    assert out[6, 2] == 1  # within the guard band of the bound
    assert out[7, 0] == orc.ABOVE_MAX and out[8, 0] == orc.OK
    assert list(out[9:, 0]) == [orc.INVALID] * 4
    assert bmax_price > 0
