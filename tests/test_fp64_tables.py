"""The FP64 erfcx, log and exp tables of the CUDA kernels, checked on the CPU.

The kernels evaluate erfcx(z) = exp(z^2) erfc(z) on 0 <= z < 128 from
piecewise Chebyshev interpolants, and ln y, log1p, exp and expm1 by Tang's
table-driven methods (csrc/fv_fp64_tables.h, written by
csrc/gen_fp64_tables.py).  Here the
committed header is what the generator writes, and each function, evaluated
step by step the way the kernel does (table rows located from the bits of the
argument, exactly rounded fused multiply-adds), is within its error bound of
mpmath on points the generator never looked at.
"""
import importlib.util
import os
import re
import struct

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2604_27210_gb300", "csrc")
HEADER = os.path.join(CSRC, "fv_fp64_tables.h")


def _gen():
    spec = importlib.util.spec_from_file_location("gen_fp64_tables",
                                                  os.path.join(CSRC, "gen_fp64_tables.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _table():
    src = open(HEADER).read()
    stride = int(re.search(r"#define FV_ERFCX_STRIDE (\d+)", src).group(1))
    body = src[src.index("{") + 1:src.index("};")]
    vals = [float(v) for v in body.replace("\n", " ").split(",") if v.strip()]
    return np.array(vals).reshape(-1, stride)


def _log_table():
    src = open(HEADER).read()
    j0 = int(re.search(r"#define FV_LOG_J0 (-?\d+)", src).group(1))
    ln2_hi = float(re.search(r"#define FV_LN2_HI (\S+)", src).group(1))
    ln2_lo = float(re.search(r"#define FV_LN2_LO (\S+)", src).group(1))
    body = src[src.index("kLogTable"):]
    body = body[body.index("{") + 1:body.index("};")]
    vals = [float(v) for v in body.replace("\n", " ").split(",") if v.strip()]
    return j0, ln2_hi, ln2_lo, np.array(vals).reshape(-1, 4)


def _log64(y, tab, corr=None):
    """The kernel's log64 for a positive normal y, operation by operation;
    with corr, ln(y + corr) (the correction enters r)."""
    j0, ln2_hi, ln2_lo, rows = tab
    bits = struct.unpack("<q", struct.pack("<d", y))[0]
    hi, lo = bits >> 32, bits & 0xffffffff
    mant = hi & 0xfffff
    m = (hi >> 20) - 1023
    if mant >= 0x6a09e:
        m += 1
        j = ((mant + (1 << 12)) >> 13) - 128
        ehi = 0x3fe00000
    else:
        j = (mant + (1 << 11)) >> 12
        ehi = 0x3ff00000
    f = struct.unpack("<d", struct.pack("<q", ((ehi | mant) << 32) | lo))[0]
    c, L_hi, L_lo, _ = rows[j - j0]
    r = _fma(f, c, -1.0)
    if corr is not None:
        r = _fma(corr * 2.0 ** -m, c, r)
    q = _fma(r, -1.0 / 6.0, 0.2)
    for k in (-0.25, 1.0 / 3.0, -0.5):
        q = _fma(q, r, k)
    p = _fma(r * r, q, r)
    md = float(m)
    return _fma(md, ln2_hi, L_hi) + (_fma(md, ln2_lo, L_lo) + p)


def _exp_table():
    src = open(HEADER).read()
    inv = float(re.search(r"#define FV_EXP_INV_LN2_N (\S+)", src).group(1))
    hi = float(re.search(r"#define FV_EXP_LN2_N_HI (\S+)", src).group(1))
    lo = float(re.search(r"#define FV_EXP_LN2_N_LO (\S+)", src).group(1))
    body = src[src.index("kExpTable"):]
    body = body[body.index("{") + 1:body.index("};")]
    vals = [float(v) for v in body.replace("\n", " ").split(",") if v.strip()]
    return inv, hi, lo, np.array(vals).reshape(-1, 2)


def _exp64(v, tab):
    """The kernel's exp64 for -708.3 < v < 709.7, operation by operation."""
    inv, hi, lo, rows = tab
    big = 6755399441055744.0
    t = _fma(v, inv, big)
    k = int(t - big)
    kd = t - big
    r = _fma(kd, -hi, v)
    r = _fma(kd, -lo, r)
    q = _fma(r, 1.0 / 120.0, 1.0 / 24.0)
    for c in (1.0 / 6.0, 0.5):
        q = _fma(q, r, c)
    p = _fma(r * r, q, r)
    t_hi, t_lo = rows[k & 127]
    return (t_hi + _fma(t_hi, p, t_lo)) * 2.0 ** (k >> 7)


def _exp_expm1(v, tab):
    """The kernel's exp_expm1_64 for -708.3 < v < 709.7: (exp v, expm1 v)."""
    inv, hi, lo, rows = tab
    big = 6755399441055744.0
    t = _fma(v, inv, big)
    k = int(t - big)
    kd = t - big
    # |v| < 0.005 on the high word, as the kernel tests it
    if (struct.unpack("<Q", struct.pack("<d", v))[0] >> 32) & 0x7fffffff < 0x3f747ae1:
        k, kd = 0, 0.0
    r = _fma(kd, -hi, v)
    r = _fma(kd, -lo, r)
    q = _fma(r, 1.0 / 720.0, 1.0 / 120.0)
    for c in (1.0 / 24.0, 1.0 / 6.0, 0.5):
        q = _fma(q, r, c)
    p = _fma(r * r, q, r)
    t_hi, t_lo = rows[k & 127]
    sc = 2.0 ** (k >> 7)
    th, tl = t_hi * sc, t_lo * sc
    return th + _fma(th, p, tl), (th - 1.0) + _fma(th, p, tl)


def _log1p_near(u, tab):
    """x = ln(1 + u) as the status rule forms it near the money (|u| <= 1):
    y = 1 + u rounded, its exact error c (Fast2Sum), then ln(y + c)."""
    y = 1.0 + u
    c = u - (y - 1.0)
    return _log64(y, tab, corr=c)


def _piece(z):
    """The kernel's piece index, from the high word of z >= 0 alone."""
    hi = struct.unpack("<q", struct.pack("<d", z))[0] >> 32
    e = (hi >> 20) - 1023
    if e >= -1:
        return 8 + ((e + 1) << 4) + ((hi >> 16) & 15)
    return ((hi & 0xfffff) | 0x100000) >> (16 - e) if e >= -4 else 0


def test_piece_index_from_the_high_word():
    # the bit formula gives the piece whose interval holds z: floor(16 z) below
    # 1/2, binade and top four fraction bits above
    g = np.random.default_rng(4)
    edges = [k / 16 for k in range(9)] + [2.0 ** e * (1 + j / 16) for e in range(-1, 7) for j in range(16)]
    z = np.concatenate([g.uniform(0, 0.5, 20000), np.exp(g.uniform(np.log(1e-300), np.log(128), 20000)),
                        edges, np.nextafter(edges, 0), np.nextafter(edges, 200), [0.0, 5e-324, 127.99999]])
    z = z[(z >= 0) & (z < 128)]
    bounds = [k / 16 for k in range(9)] + [2.0 ** e * (1 + j / 16) for e in range(-1, 7) for j in range(1, 17)]
    for zi in z:
        k = _piece(float(zi))
        assert bounds[k] <= zi < bounds[k + 1], (zi, k)


def _fma(x, y, z):
    return float(mp.mpf(x) * mp.mpf(y) + mp.mpf(z))


def _eval(tab, z):
    row = tab[_piece(z)]  # centre, then the coefficients of v^0 .. v^8
    v = z - row[0]
    p = row[9]
    for j in range(8, 0, -1):
        p = _fma(p, v, row[j])
    return p


def test_committed_table_is_the_generators_output(tmp_path):
    out = str(tmp_path / "table.h")
    _gen().main(out=out, samples=4)
    assert open(out).read() == open(HEADER).read()


def test_table_within_one_and_a_quarter_ulp_of_erfcx():
    mp.mp.dps = 40
    tab = _table()
    g = np.random.default_rng(5)
    # random points in every piece, the piece edges and their neighbours
    edges = [k / 16 for k in range(9)] + [2.0 ** e * (1 + j / 16) for e in range(-1, 7)
                                          for j in range(16)]
    z = np.concatenate([g.uniform(0, 0.5, 300), np.exp(g.uniform(np.log(0.5), np.log(128), 1200)),
                        edges, np.nextafter(edges, 0), np.nextafter(edges, 200), [0.0, 5e-324]])
    z = z[(z >= 0) & (z < 128)]
    worst = 0.0
    for zi in z:
        ref = mp.exp(mp.mpf(zi) ** 2) * mp.erfc(mp.mpf(zi))
        worst = max(worst, abs(float((_eval(tab, float(zi)) - ref) / ref)))
    # degree-8 interpolation error (up to ~0.6 ulp) plus the Horner rounding
    assert worst <= 1.25 * 2.0 ** -52, worst


def test_log_within_one_and_a_half_ulp():
    mp.mp.dps = 40
    tab = _log_table()
    g = np.random.default_rng(6)
    y = np.concatenate([np.exp(g.uniform(-700, 700, 1500)), 1 + g.uniform(-0.02, 0.02, 500),
                        1 + np.exp(g.uniform(-36, -5, 300)), 1 - np.exp(g.uniform(-36, -5, 300)),
                        g.uniform(0.5, 2.0, 1000), [1.0, 2.0, 0.5, np.sqrt(2), 2.2250738585072014e-308,
                                                     1.7976931348623157e308]])
    worst = 0.0
    for yi in y:
        ref = mp.log(mp.mpf(float(yi)))
        if ref == 0:
            assert _log64(float(yi), tab) == 0.0
            continue
        worst = max(worst, abs(float((_log64(float(yi), tab) - ref) / ref)))
    # final rounding (1/2 ulp) plus the second sum's rounding relative to a
    # result that can be as small as ln(1 + 1/256)
    assert worst <= 1.5 * 2.0 ** -52, worst


def test_exp_within_one_ulp():
    mp.mp.dps = 40
    tab = _exp_table()
    # the split head of ln2/128 has 35 significant bits: k ln2_128_hi is exact for |k| < 2^18
    hi = tab[1]
    assert (int(hi * 2 ** 42) == hi * 2 ** 42) and abs(int(hi * 2 ** 42)) < 2 ** 35
    g = np.random.default_rng(7)
    v = np.concatenate([g.uniform(-708.3, 709.7, 2000), g.uniform(-1e-3, 1e-3, 500),
                        g.uniform(-1, 1, 500), [0.0, 1.0, -1.0, 709.69, -708.29]])
    worst = 0.0
    for vi in v:
        ref = mp.exp(mp.mpf(float(vi)))
        worst = max(worst, abs(float((_exp64(float(vi), tab) - ref) / ref)))
    assert worst <= 2.0 ** -52, worst



def test_expm1_and_exp_from_one_reduction_within_one_ulp():
    mp.mp.dps = 40
    tab = _exp_table()
    g = np.random.default_rng(8)
    ln2_256 = float(np.log(2) / 256)
    # the status rule's range (v = -|x|/2 <= 0) densely, the reduction's
    # boundaries k = 0, +-1 and the binades m = -1, -2, and positive v
    v = np.concatenate([-np.exp(g.uniform(np.log(1e-300), np.log(708), 2500)),
                        g.uniform(-3 * ln2_256, 3 * ln2_256, 2000), g.uniform(-1.5, 1.5, 800),
                        g.uniform(0.0, 709.6, 500), np.exp(g.uniform(-30, 0, 300)),
                        [0.0, -0.0, ln2_256, -ln2_256, -np.log(2.0), -2 * np.log(2.0), -708.29]])
    worst_e = worst_m = 0.0
    for vi in v:
        e, m1 = _exp_expm1(float(vi), tab)
        x = mp.mpf(float(vi))
        worst_e = max(worst_e, abs(float((e - mp.exp(x)) / mp.exp(x))))
        if vi == 0:
            assert m1 == 0.0
            continue
        worst_m = max(worst_m, abs(float((m1 - mp.expm1(x)) / mp.expm1(x))))
    assert worst_e <= 2.0 ** -52, worst_e
    # the first sum exact (m = 0, -1) or half an ulp of a result beyond 1/2,
    # the second one small: about one ulp
    assert worst_m <= 1.2 * 2.0 ** -52, worst_m


def test_log1p_near_the_money_within_one_and_a_half_ulp():
    mp.mp.dps = 40
    tab = _log_table()
    g = np.random.default_rng(9)
    u = np.concatenate([g.uniform(-0.5, 1.0, 1500), np.exp(g.uniform(np.log(1e-300), 0, 800)),
                        -np.exp(g.uniform(np.log(1e-300), np.log(0.5), 800)),
                        g.uniform(-4.0 / 256, 4.0 / 256, 800), [0.0, -0.5, 1.0, 1.0 / 512, -1.0 / 512]])
    worst = 0.0
    for ui in u:
        got = _log1p_near(float(ui), tab)
        ref = mp.log1p(mp.mpf(float(ui)))
        if ref == 0:
            assert got == 0.0
            continue
        worst = max(worst, abs(float((got - ref) / ref)))
    assert worst <= 1.5 * 2.0 ** -52, worst


def _f32_trunc(d):
    """FP64 -> FP32 with the fraction truncated (the kernels' f32_trunc)."""
    hi = struct.unpack("<Q", struct.pack("<d", d))[0] >> 32
    lo = struct.unpack("<Q", struct.pack("<d", d))[0] & 0xffffffff
    e = ((hi >> 20) & 0x7ff) - 896
    sign = hi & 0x80000000
    frac = ((hi & 0xfffff) << 3) | (lo >> 29)
    bits = sign if e <= 0 else (sign | 0x7f800000 if e >= 255 else sign | (e << 23) | frac)
    return np.frombuffer(struct.pack("<I", bits), dtype=np.float32)[0]


def _piece_w(w):
    """The kernel's piece index for erfcx(w/sqrt2), w >= 0: from the FP32 view
    z_f = trunc32(w) * 0.70710677f (None: the asymptotic branch)."""
    zf = np.float32(_f32_trunc(w) * np.float32(0.70710677))
    b = struct.unpack("<I", struct.pack("<f", zf))[0]
    if b >= 0x43000000:
        return None
    e = (b >> 23) - 127
    if e >= -1:
        return 8 + ((e + 1) << 4) + ((b >> 19) & 15)
    return ((b & 0x7fffff) | 0x800000) >> (19 - e) if e >= -4 else 0


def test_w_form_piece_index_and_accuracy_next_to_edges():
    # erfcx(w/sqrt2): the FP32 view may put z = w/sqrt2 in the neighbouring
    # piece within ~2^-22 z of an edge; there the interpolant, taken that little
    # outside its interval (v = w/sqrt2 - c by one FMA), keeps its accuracy
    mp.mp.dps = 40
    tab = _table()
    bounds = [k / 16 for k in range(9)] + [2.0 ** e * (1 + j / 16) for e in range(-1, 7) for j in range(1, 17)]
    edges = np.array(bounds[1:])
    rt2 = float(np.sqrt(2.0))
    g = np.random.default_rng(11)
    w = np.concatenate([edges * rt2, np.nextafter(edges * rt2, 0), np.nextafter(edges * rt2, 1e3),
                        edges * rt2 * (1 - 2e-7), edges * rt2 * (1 + 2e-7),
                        g.uniform(0, 181, 300), [0.0, 5e-324]])
    inv_rt2 = float(1 / mp.sqrt(2))
    worst_ext = worst = 0.0
    for wi in w:
        wi = float(wi)
        k = _piece_w(wi)
        z = mp.mpf(wi) / mp.sqrt(2)
        if k is None:
            assert z > 127.99
            continue
        assert 0 <= k <= 135
        a, b = bounds[k], bounds[k + 1]
        ext = max(float(a - z), float(z - b), 0.0) / max(float(z), 1e-300)
        worst_ext = max(worst_ext, ext)
        row = tab[k]
        v = _fma(wi, inv_rt2, -row[0])
        p = row[9]
        for j in range(8, 0, -1):
            p = _fma(p, v, row[j])
        ref = mp.exp(z * z) * mp.erfc(z)
        worst = max(worst, abs(float((p - ref) / ref)))
    assert worst_ext <= 3e-7, worst_ext
    # the table's 1.25 ulp plus the rounded constant 1/sqrt2 inside v
    assert worst <= 2.0 * 2.0 ** -52, worst


def _b_exact(x, s):
    """b(x, s) for the call, x <= 0, from mpmath at 40 digits."""
    x, s = mp.mpf(x), mp.mpf(s)
    return mp.exp(x / 2) * mp.ncdf(x / s + s / 2) - mp.exp(-x / 2) * mp.ncdf(x / s - s / 2)


def test_value_past_the_inflection_point_from_the_complement():
    # e exp((h+t)^2/2) = e^{ht} = e^{x/2} = b_max, so past the inflection point
    # (h + t > 0) b = b_max - e [erfcx((h+t)/sqrt2) + erfcx((t-h)/sqrt2)]/2
    mp.mp.dps = 40
    g = np.random.default_rng(12)
    for _ in range(300):
        x = -float(np.exp(g.uniform(np.log(1e-4), np.log(30))))
        sc = (2 * -x) ** 0.5
        s = sc * float(g.uniform(1.0001, 8.0))
        X, S = mp.mpf(x), mp.mpf(s)
        h, t = X / S, S / 2
        e = mp.exp(-(h * h + t * t) / 2)
        C = (mp.exp(((h + t) / mp.sqrt(2)) ** 2) * mp.erfc((h + t) / mp.sqrt(2))
             + mp.exp(((t - h) / mp.sqrt(2)) ** 2) * mp.erfc((t - h) / mp.sqrt(2))) / 2
        b = mp.exp(X / 2) - e * C
        ref = _b_exact(x, s)
        assert abs((b - ref) / ref) < mp.mpf(10) ** -30, (x, s)


def test_lowest_region_erfcx_difference_moves_s_by_eps_over_x():
    # In the lowest region the objective is ln b.  For small t the erfcx
    # difference loses a factor ~|x|/s^2 to cancellation; with FP64 erfcx
    # values (error 1 ulp each) the error reaches ln b as an absolute error,
    # which moves s by that error over s (ln b)'.  For |x| >= 1 that is within
    # a few eps, the claim behind taking the difference there.
    mp.mp.dps = 40
    eps = 2.0 ** -52

    def worst_shift(x_lo, x_hi, n, seed):
        g = np.random.default_rng(seed)
        worst = 0.0
        for _ in range(n):
            x = -float(np.exp(g.uniform(np.log(x_lo), np.log(x_hi))))
            s = float(np.exp(g.uniform(np.log(1e-3), np.log(0.2))))
            X, S = mp.mpf(x), mp.mpf(s)
            h, t = X / S, S / 2
            z1, z2 = -(h + t) / mp.sqrt(2), (t - h) / mp.sqrt(2)
            y1 = mp.exp(z1 * z1) * mp.erfc(z1)
            y2 = mp.exp(z2 * z2) * mp.erfc(z2)
            # each FP64 erfcx value one ulp off, in the directions that add up
            lnb_true = mp.log((y1 - y2) / 2)
            lnb_fp = mp.log((y1 * (1 + eps) - y2 * (1 - eps)) / 2)
            dlnb = mp.diff(lambda ss: mp.log(_b_exact(x, ss)), S)
            worst = max(worst, float(abs((lnb_fp - lnb_true) / (S * dlnb)) / eps))
        return worst

    assert worst_shift(1.0, 20.0, 300, 13) < 4.0
    # near the money the same difference would move s by hundreds of eps:
    # there the series stays
    assert worst_shift(1e-3, 0.1, 60, 14) > 100.0
