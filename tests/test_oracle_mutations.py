"""The oracle's pins catch plausible mistakes.

Each case below plants one mistake (a dropped term, a wrong sign, a wrong
index or operand) in a copy of the oracle's sources (``oracle/fv_oracle.c``
and ``oracle/lbr_steps.h``), builds the copy with
the oracle's own flags, and runs the pins of ``tests/test_oracle.py`` against
it: at least one pin must fail.  The mistakes are made on the CPU, in the
oracle only.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_DIR = os.path.join(ROOT, "oracle")

# (what the mistake is, exact text in the oracle's sources, the mistaken text)
MUTANTS = [
    # normalised Black and price (Section 2.2 normalisation, Section 2.4)
    ("normalised Black: wrong sign of the strike term",
     "- em * Phi_q((q128)th * (h - t))", "+ em * Phi_q((q128)th * (h - t))"),
    ("normalised Black: h - t in the forward term",
     "ep * Phi_q((q128)th * (h + t))", "ep * Phi_q((q128)th * (h - t))"),
    ("erfcx: reflection with exp(-z^2)",
     "if (z < 0) return 2 * expf128(z * z) - erfcx_q(-z);",
     "if (z < 0) return 2 * expf128(-z * z) - erfcx_q(-z);"),
    ("erfcx: asymptotic series with (2k+1)!!",
     "term *= -(2 * k - 1) * v;", "term *= -(2 * k + 1) * v;"),
    ("complement: wrong sign in the second tail",
     "expf128(-0.5f128 * x) * Phi_q(h - t);", "expf128(-0.5f128 * x) * Phi_q(t - h);"),
    ("normal density: dropped factor 1/2 in the exponent",
     "q_inv_sqrt_2pi() * expf128(-0.5f128 * z * z)", "q_inv_sqrt_2pi() * expf128(-z * z)"),
    ("price: discount factor with the wrong sign",
     "q128 D = expf128(-(q128)r * (q128)T);", "q128 D = expf128((q128)r * (q128)T);"),
    ("price: forward grows with r + q",
     "(q128)SF * expf128(((q128)r - qq) * (q128)T);", "(q128)SF * expf128(((q128)r + qq) * (q128)T);"),
    ("FP64 textbook price: d2 = d1 + s",
     "d2 = d1 - s;", "d2 = d1 + s;"),
    # normalisation of a quote and the status rule
    ("normalisation: BSM log-forward with r + q",
     "*x = logf128((q128)SF / (q128)K) + ((q128)r - qq) * (q128)T;",
     "*x = logf128((q128)SF / (q128)K) + ((q128)r + qq) * (q128)T;"),
    ("normalisation: beta not undiscounted",
     "*beta = (q128)P * expf128((q128)r * (q128)T) / sqrtf128((q128)SF * (q128)K);",
     "*beta = (q128)P / sqrtf128((q128)SF * (q128)K);"),
    ("status: log-moneyness relative to the spot instead of the strike",
     "lm = log1p((SF - K) / K);", "lm = log1p((SF - K) / SF);"),
    ("status: FP64 forward with r + q",
     "x = lm + (r - qq) * T;", "x = lm + (r + qq) * T;"),
    ("status: intrinsic value with (1 - Em)",
     "const R iota = itm ? (-E * (1.0 + Em)) / Em : 0.0;\n  o->x = x;",
     "const R iota = itm ? (-E * (1.0 - Em)) / Em : 0.0;\n  o->x = x;"),
    ("status: upper band on the wrong side",
     "if (beta_otm >= bmax_otm * (1.0 - EPS_S)) {", "if (beta_otm >= bmax_otm * (1.0 + EPS_S)) {"),
    ("status: band of 4 units of 2^-52 instead of 64",
     "#define EPS_S (64.0 * 2.220446049250313080847263336181640625e-16)",
     "#define EPS_S (4.0 * 2.220446049250313080847263336181640625e-16)"),
    ("status: below-intrinsic test without its band",
     "if (beta < iota * (1.0 - EPS_S)) {", "if (beta < iota) {"),
    ("status: at-intrinsic test without its band",
     "o->solve = beta_otm > iota * EPS_S;", "o->solve = beta_otm > 0.0;"),
    ("status: in-the-money test with the wrong sign",
     "const int itm = th * x > 0;\n  const R iota = itm ? (-E * (1.0 + Em)) / Em : 0.0;\n  o->x",
     "const int itm = th * x < 0;\n  const R iota = itm ? (-E * (1.0 + Em)) / Em : 0.0;\n  o->x"),
    # conditioning (normalised vega, kappa) and the status margin: the
    # quantities the parity tests gate and excuse quotes with
    ("conditioning: kappa without the factor s",
     "c->out2[i] = (double)(beta / (s * v));", "c->out2[i] = (double)(beta / v);"),
    ("conditioning: kappa with t = s/2 for s",
     "c->out2[i] = (double)(beta / (s * v));", "c->out2[i] = (double)(beta / (t * v));"),
    ("conditioning: normalised vega with t^2 of the wrong sign",
     "q128 v = q_inv_sqrt_2pi() * expf128(-0.5f128 * (h * h + t * t));",
     "q128 v = q_inv_sqrt_2pi() * expf128(-0.5f128 * (h * h - t * t));"),
    ("conditioning: normalised vega without 1/sqrt(2 pi)",
     "q128 v = q_inv_sqrt_2pi() * expf128(-0.5f128 * (h * h + t * t));",
     "q128 v = expf128(-0.5f128 * (h * h + t * t));"),
    ("status margin: below-intrinsic threshold without its band",
     "m = fmin(m, fabs(beta / (iota * (1.0 - EPS_S)) - 1.0));", "m = fmin(m, fabs(beta / iota - 1.0));"),
    ("status margin: at-intrinsic threshold on the wrong side of the band",
     "m = fmin(m, fabs(beta / (iota * (1.0 + EPS_S)) - 1.0));",
     "m = fmin(m, fabs(beta / (iota * (1.0 - EPS_S)) - 1.0));"),
    ("status margin: upper threshold without its band",
     "fabs(beta_otm / (bmax_otm * (1.0 - EPS_S)) - 1.0)", "fabs(beta_otm / bmax_otm - 1.0)"),
    ("status margin: in-the-money bound distance not relative to beta",
     "* (bmax_otm / (beta > bmax_otm ? beta : bmax_otm))", ""),
    ("status margin: not in units of 2^-52",
     "return m / eps;", "return m;"),
    # the definition of implied volatility
    ("definition: bisection keeps the wrong half",
     "    if (nb_q_e(x, mid, 1, ep, em) < beta)\n      lo = mid;",
     "    if (nb_q_e(x, mid, 1, ep, em) > beta)\n      lo = mid;"),
    ("definition: intrinsic value not removed in the money",
     "q128 beta_otm = ((q128)th * x > 0) ? beta - iota : beta;", "q128 beta_otm = beta;"),
    # the oracle's FP64 normalised Black (the CPU baseline's evaluation)
    ("FP64 normalised Black: Mills-ratio recurrence with k for k + 1",
     "const R R3 = (k + 1) * Rk + h * R2;", "const R R3 = k * Rk + h * R2;"),
    ("FP64 erfcx: continued fraction with partial numerators k for k/2",
     "const double a = 0.5 * k;", "const double a = 1.0 * k;"),
    ("FP64 normalised Black: CDF-direct form with the wrong sign",
     "if (cdf_direct(h, t)) return exp(0.5 * x) * Phi_d(h + t) - exp(-0.5 * x) * Phi_d(h - t);",
     "if (cdf_direct(h, t)) return exp(0.5 * x) * Phi_d(h + t) + exp(-0.5 * x) * Phi_d(h - t);"),
    ("FP64 normalised Black: ln b with +ln sqrt(2 pi)",
     "*L = log(D) - 0.5 * (h * h + t * t) - LN_SQRT_2PI;",
     "*L = log(D) - 0.5 * (h * h + t * t) + LN_SQRT_2PI;"),
    ("FP64 erfcx: exp(-z^2) for exp(z^2)",
     "if (z < 2.0) return exp(z * z) * erfc(z);", "if (z < 2.0) return exp(-z * z) * erfc(z);"),
    ("FP64 complement: wrong sign in the second tail",
     "return exp(0.5 * x) * Phi_d(-(h + t)) + exp(-0.5 * x) * Phi_d(h - t);",
     "return exp(0.5 * x) * Phi_d(-(h + t)) + exp(-0.5 * x) * Phi_d(t - h);"),
    # Let's Be Rational, step by step
    ("LBR: normalised vega with t^2 of the wrong sign",
     "return exp(-0.5 * (h * h + t * t)) * INV_SQRT_2PI;", "return exp(-0.5 * (h * h - t * t)) * INV_SQRT_2PI;"),
    ("LBR: lowest-wing guess with a square root for the cube root",
     "Phi_inv_d(cbrt(beta / cl))", "Phi_inv_d(sqrt(beta / cl))"),
    ("LBR: Hermite guess with swapped end slopes",
     "s = hermite_guess(beta, bc, bh, sc, sh, 1.0 / vc, 1.0 / vh);",
     "s = hermite_guess(beta, bc, bh, sc, sh, 1.0 / vh, 1.0 / vc);"),
    ("LBR: upper objective derivative without w",
     "h2 = u + w;\n      h3 = h2 * h2 + du + w * h2;", "h2 = u;\n      h3 = h2 * h2 + du + w * h2;"),
    ("LBR: lowest objective derivative with 1 - 2/L",
     "const R k1 = 1.0 + 2.0 / L;", "const R k1 = 1.0 - 2.0 / L;"),
    ("LBR: Householder step without the h3 term",
     "R ds = nu * (1.0 + 0.5 * h2 * nu) / (1.0 + nu * (h2 + h3 * nu / 6.0));",
     "R ds = nu * (1.0 + 0.5 * h2 * nu) / (1.0 + nu * h2);"),
    ("LBR: middle residual with the wrong sign",
     "nu = -(b - beta) / bp;", "nu = (b - beta) / bp;"),
    ("LBR: b''/b' = x^2/s^3 + s/4",
     "const R u = h * h / s - 0.25 * s;           /* b''/b' */",
     "const R u = h * h / s + 0.25 * s;           /* b''/b' */"),
    # Halley and its fallback
    ("Halley: residual b - beta with the wrong sign",
     "const double g = upper ? (bmax - beta) - nbc_d(x, s) : nb_d(x, s) - beta;",
     "const double g = upper ? (bmax - beta) - nbc_d(x, s) : beta - nb_d(x, s);"),
    ("Halley fallback: transformed residual with the wrong sign",
     "return inv_ln_beta - 1.0 / L;", "return 1.0 / L - inv_ln_beta;"),
    # Greeks and the gradient
    ("Greeks: theta without the sign change",
     "c->out4[i] = (double)(-p.dT / 365.0f128);", "c->out4[i] = (double)(p.dT / 365.0f128);"),
    ("Greeks: vega not per 1 %",
     "c->out3[i] = (double)(p.vega * 0.01f128);", "c->out3[i] = (double)(p.vega);"),
    ("Greeks: BSM theta without the r K term",
     " + qth * qr * qK * Dr * N2;", ";"),
    ("Greeks: Black-76 rho with the wrong sign",
     "o->dr = -qT * o->V;", "o->dr = qT * o->V;"),
    ("Greeks: gamma divided by S instead of S sigma sqrt(T)",
     "o->gamma = Dq * n1 / (S * sv);", "o->gamma = Dq * n1 / S;"),
    ("gradient: d sigma / d K with the wrong sign",
     "c->out3[i] = (double)(-g * p.dK / p.vega);", "c->out3[i] = (double)(g * p.dK / p.vega);"),
    ("gradient: d sigma / d q from the dividend partial of another input",
     "c->out6[i] = (double)(-g * p.dq / p.vega);", "c->out6[i] = (double)(-g * p.dr / p.vega);"),
]


# the oracle's sources; a mistake is planted in the one that holds its text
SOURCES = ("fv_oracle.c", "lbr_steps.h")


def _pins_fail_with(what, old, new, workdir):
    """Build the oracle with one mistake planted; True when a pin fails."""
    from oracle import build as obuild
    srcs = {name: open(os.path.join(ORACLE_DIR, name)).read() for name in SOURCES}
    hits = [name for name in SOURCES if old in srcs[name]]
    assert len(hits) == 1 and srcs[hits[0]].count(old) == 1, \
        "the text to mutate must occur exactly once: %r" % old
    srcs[hits[0]] = srcs[hits[0]].replace(old, new)
    os.makedirs(workdir)
    for name, text in srcs.items():
        with open(os.path.join(workdir, name), "w") as f:
            f.write(text)
    shutil.copy(os.path.join(ORACLE_DIR, "fv_oracle.h"), workdir)
    lib = os.path.join(workdir, "liboracle_mutant.so")
    obuild.compile_library([os.path.join(workdir, "fv_oracle.c")], lib)
    env = dict(os.environ, FV_ORACLE_LIB=lib, PYTHONDONTWRITEBYTECODE="1", OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle.py"),
                        "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode == 1, r.stdout[-1500:]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    # the mutants run concurrently, each in its own pytest process
    workers = max(1, min(len(MUTANTS), (os.cpu_count() or 2) // 2))
    with ThreadPoolExecutor(workers) as pool:
        results = list(pool.map(lambda k: _pins_fail_with(*MUTANTS[k], str(tmp_path / str(k))),
                                range(len(MUTANTS))))
    survivors = ["%s\n%s" % (MUTANTS[k][0], out) for k, (caught, out) in enumerate(results)
                 if not caught]
    assert not survivors, "no pin caught:\n" + "\n\n".join(survivors)


def test_the_harness_passes_the_unchanged_oracle(tmp_path):
    # control: the same copy-build-run path with nothing planted passes every pin
    same = MUTANTS[0][1]
    failed, out = _pins_fail_with("control", same, same, str(tmp_path / "control"))
    assert not failed, out
