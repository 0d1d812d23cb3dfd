"""The C ABI without a GPU: libfv.so loads, exports every symbol include/fv.h
declares, and rejects bad arguments before any CUDA call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fv.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2604_27210_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fv_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("fv_price", "fv_implied_vol", "fv_greeks", "fv_iv_adjoint", "fv_implied_vol_ex",
                 "fv_chains_plan_create", "fv_implied_vol_chains", "fv_chains_plan_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_lists_every_declared_symbol():
    from paper_2604_27210_gb300 import fv
    assert sorted(fv.EXPORTS) == declared_symbols()


def declared_constants():
    """Every enumerator and #define FV_* value of the header, by name."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    consts = {}
    for body in re.findall(r"typedef\s+enum\s*\{(.*?)\}", src, flags=re.S):
        for name, value in re.findall(r"\b(FV_[A-Z0-9_]+)\s*=\s*(-?\d+)", body):
            consts[name] = int(value)
    for name, value in re.findall(r"#define\s+(FV_[A-Z0-9_]+)\s+(-?\d+)", src):
        consts[name] = int(value)
    return consts


def test_binding_constants_match_the_header():
    # the Python names of the enumerators carry the header's values (an enum
    # the binding does not name is fine; a wrong value is not)
    from paper_2604_27210_gb300 import fv
    consts = declared_constants()
    for must in ("FV_BSM", "FV_HALLEY", "FV_FP32", "FV_DTYPE_F32", "FV_TRANSFER_DIRECT",
                 "FV_NOALLOC_MAX_QUOTES", "FV_ERR_ARG"):
        assert must in consts, must
    named = {k: v for k, v in consts.items() if hasattr(fv, k)}
    assert len(named) >= 20, sorted(named)
    for k, v in named.items():
        assert getattr(fv, k) == v, (k, getattr(fv, k), v)


def _p(v=0x1000):
    return ctypes.c_void_p(v)


def test_argument_errors_before_any_launch(lib):
    lib.fv_implied_vol.restype = ctypes.c_int
    lib.fv_last_error.restype = ctypes.c_char_p
    N = ctypes.c_int64
    p = _p()
    # unknown model / solver, n < 0, NULL required pointers, BSM without q
    assert lib.fv_implied_vol(9, 0, p, p, p, p, p, None, p, N(4), p, p, None) == -1
    assert b"unknown model" in lib.fv_last_error()
    assert lib.fv_implied_vol(0, 9, p, p, p, p, p, None, p, N(4), p, p, None) == -1
    assert lib.fv_implied_vol(0, 0, p, p, p, p, p, None, p, N(-3), p, p, None) == -1
    assert b"n = -3" in lib.fv_last_error()
    assert lib.fv_implied_vol(0, 0, p, None, p, p, p, None, p, N(4), p, p, None) == -1
    assert b"S_or_F" in lib.fv_last_error()
    assert lib.fv_implied_vol(2, 0, p, p, p, p, p, None, p, N(4), p, p, None) == -1
    assert b"q is NULL" in lib.fv_last_error()
    # n = 0 is valid and touches nothing, even with NULL pointers
    assert lib.fv_implied_vol(0, 0, None, None, None, None, None, None, None, N(0), None, None,
                              None) == 0
    lib.fv_price.restype = ctypes.c_int
    assert lib.fv_price(5, p, p, p, p, p, None, p, N(1), p, None) == -1
    lib.fv_greeks.restype = ctypes.c_int
    assert lib.fv_greeks(0, p, p, p, p, p, None, p, N(-1), p, p, p, p, p, None) == -1
    lib.fv_iv_adjoint.restype = ctypes.c_int
    assert lib.fv_iv_adjoint(0, None, p, p, p, p, None, p, p, p, p, N(2), p, p, p, p, p, p,
                             None) == -1  # Black-76 adjoint needs the price
    lib.fv_implied_vol_ex.restype = ctypes.c_int
    assert lib.fv_implied_vol_ex(0, 0, 7, 0, p, p, p, p, p, None, p, N(4), p, p, None) == -1
    assert lib.fv_implied_vol_ex(0, 0, 0, 5, p, p, p, p, p, None, p, N(4), p, p, None) == -1
    # the Halley solver has no mixed path
    assert lib.fv_implied_vol_ex(0, 1, 1, 0, p, p, p, p, p, None, p, N(4), p, p, None) == -3
    lib.fv_math.restype = ctypes.c_int
    assert lib.fv_math(6, p, N(4), p, None) == -1
    assert b"unknown function" in lib.fv_last_error()
    assert lib.fv_math(4, p, N(-1), p, None) == -1
    assert lib.fv_math(3, None, N(4), p, None) == -1
    assert lib.fv_math(4, None, N(0), None, None) == 0


def test_workspace_size_and_checks(lib):
    lib.fv_workspace_size.restype = ctypes.c_size_t
    lib.fv_workspace_size.argtypes = [ctypes.c_int, ctypes.c_int64]
    assert lib.fv_workspace_size(0, 1000) == 0
    need = lib.fv_workspace_size(1, 1000)
    assert need >= 1000 * 20
    lib.fv_implied_vol_ws.restype = ctypes.c_int
    N = ctypes.c_int64
    p = _p()
    # too small, NULL and misaligned workspaces are argument errors
    assert lib.fv_implied_vol_ws(0, 1, p, p, p, p, p, None, p, N(1000), p, p, p,
                                 ctypes.c_size_t(need - 1), None) == -1
    assert lib.fv_implied_vol_ws(0, 1, p, p, p, p, p, None, p, N(1000), p, p, None,
                                 ctypes.c_size_t(need), None) == -1
    assert lib.fv_implied_vol_ws(0, 1, p, p, p, p, p, None, p, N(1000), p, p, _p(0x1008),
                                 ctypes.c_size_t(need), None) == -1


def test_chains_plan_argument_errors(lib):
    from paper_2604_27210_gb300.fv import fv_chain
    lib.fv_chains_plan_create.restype = ctypes.c_int
    h = ctypes.c_void_p()
    arr = (fv_chain * 2)()
    arr[0].n = 5
    arr[1].n = -1
    assert lib.fv_chains_plan_create(0, 0, arr, ctypes.c_int64(2), 0, None, ctypes.byref(h)) == -1
    assert lib.fv_chains_plan_create(0, 1, arr, ctypes.c_int64(2), 0, None, ctypes.byref(h)) == -3
    assert lib.fv_chains_plan_create(0, 0, None, ctypes.c_int64(-1), 0, None, ctypes.byref(h)) == -1
    lib.fv_chains_plan_destroy.restype = ctypes.c_int
    assert lib.fv_chains_plan_destroy(None) == 0


def test_status_strings(lib):
    lib.fv_status_string.restype = ctypes.c_char_p
    for code, word in ((0, b"SUCCESS"), (-1, b"ARG"), (-2, b"CUDA"), (-3, b"UNSUPPORTED"),
                       (-4, b"NOMEM")):
        assert word in lib.fv_status_string(code)


def test_autotune_cache_round_trip(tmp_path):
    # the chains plan's tuning cache is host code: seeded, read back, replaced
    # and rejected keys, all without a GPU
    from paper_2604_27210_gb300 import fv
    path = str(tmp_path / "tune.json")
    key = "NVIDIA GB300|sm152|model0|chains2^13|quotes2^26|len2^12"
    assert fv.fv_autotune_cache_get(path, key) is None  # no file yet
    fv.fv_autotune_cache_put(path, key, 128, 2, 6, 35.5)
    fv.fv_autotune_cache_put(path, "other|sm1", 512, 1, 1, 1.25)
    assert fv.fv_autotune_cache_get(path, key) == dict(block=128, quotes_per_thread=2,
                                                       blocks_per_sm=6, ms=35.5)
    fv.fv_autotune_cache_put(path, key, 256, 4, 2, 30.0)  # replaced, the other entry kept
    assert fv.fv_autotune_cache_get(path, key)["block"] == 256
    assert fv.fv_autotune_cache_get(path, "other|sm1")["quotes_per_thread"] == 1
    import json
    with open(path) as f:
        assert set(json.load(f)) == {key, "other|sm1"}  # the file is plain JSON
    for bad in ('quote"d', "", "line\nbreak"):
        with pytest.raises(fv.FvError):
            fv.fv_autotune_cache_put(path, bad, 256, 2, 1, 1.0)
    with pytest.raises(fv.FvError):
        fv.fv_autotune_cache_put(path, "k", 0, 2, 1, 1.0)


def test_fv_log_reports_calls_and_errors():
    # FV_LOG=1: the entry point's name and batch size, and the argument error,
    # on stderr (argument errors precede any CUDA call, so no GPU is needed)
    import subprocess
    import sys
    code = ("import ctypes; from paper_2604_27210_gb300 import build; "
            "lib = ctypes.CDLL(build.build()); p = ctypes.c_void_p(0x1000); "
            "rc = lib.fv_implied_vol(0, 0, p, None, p, p, p, None, p, ctypes.c_int64(4), p, p, None); "
            "print(rc)")
    env = dict(os.environ, FV_LOG="1")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.stdout.strip() == "-1", r.stderr
    assert "fv: fv_implied_vol n=4" in r.stderr
    assert "fv: error -1: fv_implied_vol: S_or_F is NULL" in r.stderr
    env["FV_LOG"] = "0"
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=120)
    assert "fv:" not in r.stderr
