"""ctypes wrapper of the C oracle (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  Every function takes and returns host
numpy arrays; model codes are 0 Black-76, 1 Black-Scholes, 2 BSM; status codes
are 0 OK, 1 below intrinsic, 2 above maximum, 3 invalid.

FV_ORACLE_LIB=<path> loads another build of the same C source instead of
``oracle/_build/liboracle.so`` (the planted-mistake tests point it at copies
of the oracle with one mistake each).
"""
import ctypes
import os

import numpy as np

from . import build as _build

BLACK76, BLACK_SCHOLES, BSM = 0, 1, 2
OK, BELOW_INTRINSIC, ABOVE_MAX, INVALID = 0, 1, 2, 3

_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I8 = ctypes.POINTER(ctypes.c_int8)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_N = ctypes.c_int64
_INT = ctypes.c_int


def _load():
    global _lib
    if _lib is None:
        path = os.environ.get("FV_ORACLE_LIB") or _build.build()
        lib = ctypes.CDLL(path)
        lib.or_num_threads.restype = _INT
        lib.or_normalised_black.argtypes = [_D, _D, _I8, _N, _D, _INT]
        lib.or_erfcx.argtypes = [_D, _N, _D, _INT]
        lib.or_price.argtypes = [_INT, _D, _D, _D, _D, _D, _D, _I8, _N, _D, _INT]
        lib.or_price_f64.argtypes = [_INT, _D, _D, _D, _D, _D, _D, _I8, _N, _D, _INT]
        lib.or_status.argtypes = [_INT, _D, _D, _D, _D, _D, _D, _I8, _N, _U8, _D, _D, _D, _INT]
        lib.or_iv.argtypes = [_INT, _D, _D, _D, _D, _D, _D, _I8, _N, _D, _U8, _INT]
        lib.or_conditioning.argtypes = [_INT, _D, _D, _D, _D, _D, _D, _I8, _D, _N, _D, _D, _INT]
        lib.or_iv_lbr.argtypes = [_INT, _D, _D, _D, _D, _D, _D, _I8, _N, _INT, _D, _U8, _I8, _INT]
        lib.or_iv_lbr_f64.argtypes = [_INT, _D, _D, _D, _D, _D, _D, _I8, _N, _INT, _D, _U8, _I8,
                                      _INT]
        lib.or_normalised_black_f64.argtypes = [_D, _D, _I8, _N, _D, _INT]
        lib.or_iv_halley.argtypes = [_INT, _D, _D, _D, _D, _D, _D, _I8, _N, _D, _U8, _U8, _INT]
        lib.or_greeks.argtypes = [_INT, _D, _D, _D, _D, _D, _D, _I8, _N, _D, _D, _D, _D, _D, _INT]
        lib.or_iv_grad.argtypes = [_INT, _D, _D, _D, _D, _D, _I8, _D, _U8, _D, _N,
                                   _D, _D, _D, _D, _D, _D, _INT]
        _lib = lib
    return _lib


def num_threads() -> int:
    return _load().or_num_threads()


def _f64(a, n):
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), (n,)))
    return a, a.ctypes.data_as(_D)


def _i8(a, n):
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.int8), (n,)))
    return a, a.ctypes.data_as(_I8)


def _u8(a, n):
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.uint8), (n,)))
    return a, a.ctypes.data_as(_U8)


def _len(*arrays):
    n = 1
    for a in arrays:
        if a is not None and np.ndim(a) > 0:
            n = max(n, np.size(a))
    return n


def normalised_black(x, s, theta=1, nthreads=0):
    n = _len(x, s, theta)
    keep = [_f64(x, n), _f64(s, n), _i8(theta, n)]
    out = np.empty(n, np.float64)
    _load().or_normalised_black(keep[0][1], keep[1][1], keep[2][1], n, out.ctypes.data_as(_D),
                                nthreads)
    return out


def normalised_black_f64(x, s, theta=1, nthreads=0):
    """The oracle's own FP64 evaluation of the normalised Black function."""
    n = _len(x, s, theta)
    keep = [_f64(x, n), _f64(s, n), _i8(theta, n)]
    out = np.empty(n, np.float64)
    _load().or_normalised_black_f64(keep[0][1], keep[1][1], keep[2][1], n, out.ctypes.data_as(_D),
                                    nthreads)
    return out


def erfcx(z, nthreads=0):
    n = _len(z)
    zz = _f64(z, n)
    out = np.empty(n, np.float64)
    _load().or_erfcx(zz[1], n, out.ctypes.data_as(_D), nthreads)
    return out


def price(model, S_or_F, K, T, r, q, sigma, flag, nthreads=0):
    n = _len(S_or_F, K, T, r, q, sigma, flag)
    keep = [_f64(S_or_F, n), _f64(K, n), _f64(T, n), _f64(r, n), _f64(0.0 if q is None else q, n),
            _f64(sigma, n), _i8(flag, n)]
    out = np.empty(n, np.float64)
    _load().or_price(model, keep[0][1], keep[1][1], keep[2][1], keep[3][1], keep[4][1], keep[5][1],
                     keep[6][1], n, out.ctypes.data_as(_D), nthreads)
    return out


def price_f64(model, S_or_F, K, T, r, q, sigma, flag, nthreads=0):
    """Textbook price in plain FP64 (fast input generator for large sets)."""
    n = _len(S_or_F, K, T, r, q, sigma, flag)
    keep = [_f64(S_or_F, n), _f64(K, n), _f64(T, n), _f64(r, n), _f64(0.0 if q is None else q, n),
            _f64(sigma, n), _i8(flag, n)]
    out = np.empty(n, np.float64)
    _load().or_price_f64(model, *[k[1] for k in keep], n, out.ctypes.data_as(_D), nthreads)
    return out


def status(model, P, S_or_F, K, T, r, q, flag, nthreads=0):
    """FP64 status rule: (status, x, beta, margin to the nearest threshold in 2^-52 units)."""
    n = _len(P, S_or_F, K, T, r, q, flag)
    keep = [_f64(P, n), _f64(S_or_F, n), _f64(K, n), _f64(T, n), _f64(r, n),
            _f64(0.0 if q is None else q, n), _i8(flag, n)]
    st = np.empty(n, np.uint8)
    x = np.empty(n, np.float64)
    beta = np.empty(n, np.float64)
    margin = np.empty(n, np.float64)
    _load().or_status(model, *[k[1] for k in keep], n, st.ctypes.data_as(_U8), x.ctypes.data_as(_D),
                      beta.ctypes.data_as(_D), margin.ctypes.data_as(_D), nthreads)
    return st, x, beta, margin


def _iv_common(fn, model, P, S_or_F, K, T, r, q, flag, extra=(), nthreads=0, aux=None):
    n = _len(P, S_or_F, K, T, r, q, flag)
    keep = [_f64(P, n), _f64(S_or_F, n), _f64(K, n), _f64(T, n), _f64(r, n),
            _f64(0.0 if q is None else q, n), _i8(flag, n)]
    sig = np.empty(n, np.float64)
    st = np.empty(n, np.uint8)
    args = [model] + [k[1] for k in keep] + [n] + list(extra) + [sig.ctypes.data_as(_D),
                                                                  st.ctypes.data_as(_U8)]
    if aux is not None:
        a = np.empty(n, aux)
        args.append(a.ctypes.data_as(_I8 if aux == np.int8 else _U8))
    else:
        a = None
    args.append(nthreads)
    fn(*args)
    return sig, st, a


def iv(model, P, S_or_F, K, T, r, q, flag, nthreads=0):
    """Implied volatility by definition (binary128 bisection) and status."""
    sig, st, _ = _iv_common(_load().or_iv, model, P, S_or_F, K, T, r, q, flag, nthreads=nthreads)
    return sig, st


def iv_lbr(model, P, S_or_F, K, T, r, q, flag, n_iter=3, nthreads=0):
    """FP64 "Let's Be Rational" steps; returns sigma, status, region."""
    return _iv_common(_load().or_iv_lbr, model, P, S_or_F, K, T, r, q, flag, extra=(n_iter,),
                      nthreads=nthreads, aux=np.int8)


def iv_lbr_f64(model, P, S_or_F, K, T, r, q, flag, n_iter=3, nthreads=0):
    """The LBR steps with the oracle's FP64 normalised Black (the CPU
    baseline); returns sigma, status, region."""
    return _iv_common(_load().or_iv_lbr_f64, model, P, S_or_F, K, T, r, q, flag, extra=(n_iter,),
                      nthreads=nthreads, aux=np.int8)


def iv_halley(model, P, S_or_F, K, T, r, q, flag, nthreads=0):
    """FP64 Halley x8 + bisection fallback; returns sigma, status, fallback flag."""
    return _iv_common(_load().or_iv_halley, model, P, S_or_F, K, T, r, q, flag, nthreads=nthreads,
                      aux=np.uint8)


def conditioning(model, P, S_or_F, K, T, r, q, flag, sigma, nthreads=0):
    """Normalised vega b'(x, s) and kappa = beta / (s b') at sigma."""
    n = _len(P, S_or_F, K, T, r, q, flag, sigma)
    keep = [_f64(P, n), _f64(S_or_F, n), _f64(K, n), _f64(T, n), _f64(r, n),
            _f64(0.0 if q is None else q, n), _i8(flag, n), _f64(sigma, n)]
    v = np.empty(n, np.float64)
    k = np.empty(n, np.float64)
    _load().or_conditioning(model, *[a[1] for a in keep], n, v.ctypes.data_as(_D),
                            k.ctypes.data_as(_D), nthreads)
    return v, k


def greeks(model, S_or_F, K, T, r, q, sigma, flag, nthreads=0):
    """(delta, gamma, vega, theta, rho) in the py_vollib scaling."""
    n = _len(S_or_F, K, T, r, q, sigma, flag)
    keep = [_f64(S_or_F, n), _f64(K, n), _f64(T, n), _f64(r, n), _f64(0.0 if q is None else q, n),
            _f64(sigma, n), _i8(flag, n)]
    outs = [np.empty(n, np.float64) for _ in range(5)]
    _load().or_greeks(model, *[a[1] for a in keep], n, *[o.ctypes.data_as(_D) for o in outs],
                      nthreads)
    return tuple(outs)


def iv_grad(model, S_or_F, K, T, r, q, flag, sigma, status_, grad_sigma, nthreads=0):
    """(gP, gS, gK, gT, gr, gq): grad_sigma times d sigma / d input."""
    n = _len(S_or_F, K, T, r, q, flag, sigma, status_, grad_sigma)
    keep = [_f64(S_or_F, n), _f64(K, n), _f64(T, n), _f64(r, n), _f64(0.0 if q is None else q, n),
            _i8(flag, n), _f64(sigma, n), _u8(status_, n), _f64(grad_sigma, n)]
    outs = [np.empty(n, np.float64) for _ in range(6)]
    _load().or_iv_grad(model, *[a[1] for a in keep], n, *[o.ctypes.data_as(_D) for o in outs],
                       nthreads)
    return tuple(outs)


__all__ = ["BLACK76", "BLACK_SCHOLES", "BSM", "OK", "BELOW_INTRINSIC", "ABOVE_MAX", "INVALID",
           "normalised_black", "normalised_black_f64", "price", "price_f64", "status", "iv", "iv_lbr",
           "iv_lbr_f64", "iv_halley", "conditioning",
           "greeks", "iv_grad", "num_threads"]

if os.environ.get("FV_ORACLE_EAGER"):
    _load()
