"""Thin Python binding of libfv.so (include/fv.h), same names as the C ABI.

Argument marshalling only: tensors must already live on the GPU; every step of
the computation runs in the library's CUDA kernels.  PyTorch supplies device
memory and the current stream.  There is no CPU fallback: importing this module
without a built libfv.so raises.
"""
import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfv.so")

FV_BLACK76, FV_BLACK_SCHOLES, FV_BSM = 0, 1, 2
FV_LBR, FV_HALLEY = 0, 1
FV_FP64, FV_MIXED, FV_FP32 = 0, 1, 2
FV_DTYPE_F64, FV_DTYPE_F32 = 0, 1
FV_TRANSFER_AUTO, FV_TRANSFER_STAGED, FV_TRANSFER_DIRECT = 0, 1, 2
FV_Q_OK, FV_Q_BELOW_INTRINSIC, FV_Q_ABOVE_MAX, FV_Q_INVALID = 0, 1, 2, 3
FV_SUCCESS, FV_ERR_ARG, FV_ERR_CUDA, FV_ERR_UNSUPPORTED, FV_ERR_NOMEM = 0, -1, -2, -3, -4

# every symbol include/fv.h declares
EXPORTS = ["fv_price", "fv_implied_vol", "fv_workspace_size", "fv_implied_vol_ws",
           "fv_implied_vol_ex", "fv_implied_vol_strided", "fv_greeks", "fv_iv_adjoint",
           "fv_normalised_black", "fv_math",
           "fv_chains_plan_create", "fv_implied_vol_chains", "fv_implied_vol_chains_direct",
           "fv_chains_plan_info", "fv_chains_plan_tuning", "fv_autotune_cache_get",
           "fv_autotune_cache_put", "fv_chains_plan_destroy", "fv_stream_plan_create",
           "fv_stream_plan_destroy", "fv_stream_plan_set_transfer", "fv_stream_plan_last_transfer",
           "fv_implied_vol_host", "fv_implied_vol_halley_noalloc",
           "fv_status_string", "fv_last_error"]


class FvError(RuntimeError):
    def __init__(self, code, fn, detail):
        super().__init__("%s failed (%d): %s" % (fn, code, detail))
        self.code = code


class fv_chain(ctypes.Structure):
    _fields_ = [("price", ctypes.c_void_p), ("K", ctypes.c_void_p), ("flag", ctypes.c_void_p),
                ("sigma", ctypes.c_void_p), ("status", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("S_or_F", ctypes.c_double), ("T", ctypes.c_double), ("r", ctypes.c_double),
                ("q", ctypes.c_double)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_N = ctypes.c_int64


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libfv.so is not built (%s): run __graft_entry__.build() "
                          "or python paper_2604_27210_gb300/build.py" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    E = ctypes.c_int
    lib.fv_price.argtypes = [_I, _P, _P, _P, _P, _P, _P, _P, _N, _P, _P]
    lib.fv_implied_vol.argtypes = [_I, _I, _P, _P, _P, _P, _P, _P, _P, _N, _P, _P, _P]
    lib.fv_workspace_size.argtypes = [_I, _N]
    lib.fv_workspace_size.restype = ctypes.c_size_t
    lib.fv_implied_vol_ws.argtypes = [_I, _I, _P, _P, _P, _P, _P, _P, _P, _N, _P, _P, _P,
                                      ctypes.c_size_t, _P]
    lib.fv_implied_vol_ex.argtypes = [_I, _I, _I, _I, _P, _P, _P, _P, _P, _P, _P, _N, _P, _P, _P]
    lib.fv_implied_vol_strided.argtypes = [_I, _I, _I, _I, _P, _P, _P, _P, _P, _P, _P,
                                           ctypes.POINTER(ctypes.c_int64), _N, _P, _P, _P]
    lib.fv_greeks.argtypes = [_I, _P, _P, _P, _P, _P, _P, _P, _N, _P, _P, _P, _P, _P, _P]
    lib.fv_iv_adjoint.argtypes = [_I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _N,
                                  _P, _P, _P, _P, _P, _P, _P]
    lib.fv_normalised_black.argtypes = [_P, _P, _P, _N, _P, _P]
    lib.fv_math.argtypes = [ctypes.c_int, _P, _N, _P, _P]
    lib.fv_chains_plan_create.argtypes = [_I, _I, ctypes.POINTER(fv_chain), _N, _I, _P,
                                          ctypes.POINTER(ctypes.c_void_p)]
    lib.fv_implied_vol_chains.argtypes = [_P, _P]
    lib.fv_implied_vol_chains_direct.argtypes = [_P, _P]
    lib.fv_chains_plan_info.argtypes = [_P] + [ctypes.POINTER(_I)] * 3 + [ctypes.POINTER(_N)] * 2
    lib.fv_chains_plan_tuning.argtypes = [_P, ctypes.POINTER(_I), ctypes.POINTER(_I),
                                          ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double),
                                          ctypes.c_char_p, ctypes.c_size_t]
    lib.fv_autotune_cache_get.argtypes = [ctypes.c_char_p, ctypes.c_char_p] + \
        [ctypes.POINTER(_I)] * 3 + [ctypes.POINTER(ctypes.c_double)]
    lib.fv_autotune_cache_put.argtypes = [ctypes.c_char_p, ctypes.c_char_p, _I, _I, _I,
                                          ctypes.c_double]
    lib.fv_chains_plan_destroy.argtypes = [_P]
    lib.fv_stream_plan_create.argtypes = [_N, ctypes.POINTER(ctypes.c_void_p)]
    lib.fv_stream_plan_destroy.argtypes = [_P]
    lib.fv_stream_plan_set_transfer.argtypes = [_P, _I]
    lib.fv_stream_plan_last_transfer.argtypes = [_P, ctypes.POINTER(_I)]
    lib.fv_implied_vol_host.argtypes = [_P, _I, _I, _I, _I, _P, _P, _P, _P, _P, _P, _P, _N, _P, _P,
                                        _P]
    lib.fv_implied_vol_halley_noalloc.argtypes = [_I, _P, _P, _P, _P, _P, _P, _P, _N, _P, _P, _P]
    lib.fv_status_string.argtypes = [_I]
    lib.fv_status_string.restype = ctypes.c_char_p
    lib.fv_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("fv_workspace_size", "fv_status_string", "fv_last_error"):
            getattr(lib, name).restype = E
    return lib


_lib = _load()


def library():
    """The loaded ctypes handle of libfv.so."""
    return _lib


def _check(code, fn):
    if code != FV_SUCCESS:
        raise FvError(code, fn, _lib.fv_last_error().decode())


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t, n, dtypes, name, allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise ValueError("%s is required" % name)
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype not in dtypes:
        raise TypeError("%s has dtype %s, expected one of %s" % (name, t.dtype, dtypes))
    if not t.is_contiguous() or t.numel() != n:
        raise ValueError("%s must be contiguous with %d elements" % (name, n))
    return ctypes.c_void_p(t.data_ptr())


_F64 = (torch.float64,)
_F32 = (torch.float32,)
_I8 = (torch.int8,)
_U8 = (torch.uint8,)


def _like(t, dtype):
    return torch.empty(t.numel(), dtype=dtype, device=t.device)


def fv_price(model, flag, S_or_F, K, T, r, q, sigma, out=None, stream=None):
    n = S_or_F.numel()
    out = _like(S_or_F, torch.float64) if out is None else out
    _check(_lib.fv_price(model, _ptr(flag, n, _I8, "flag"), _ptr(S_or_F, n, _F64, "S_or_F"),
                         _ptr(K, n, _F64, "K"), _ptr(T, n, _F64, "T"), _ptr(r, n, _F64, "r"),
                         _ptr(q, n, _F64, "q", allow_none=model != FV_BSM),
                         _ptr(sigma, n, _F64, "sigma"), n, _ptr(out, n, _F64, "out"),
                         _stream(stream)), "fv_price")
    return out


def _iv_outputs(ref, out_sigma, status):
    if out_sigma is None:
        out_sigma = _like(ref, torch.float64)
    if status is None:
        status = _like(ref, torch.uint8)
    return out_sigma, status


def fv_implied_vol(model, solver, price, S_or_F, K, T, r, q, flag, out_sigma=None, status=None,
                   stream=None):
    n = price.numel()
    out_sigma, status = _iv_outputs(price, out_sigma, status)
    _check(_lib.fv_implied_vol(model, solver, _ptr(price, n, _F64, "price"),
                               _ptr(S_or_F, n, _F64, "S_or_F"), _ptr(K, n, _F64, "K"),
                               _ptr(T, n, _F64, "T"), _ptr(r, n, _F64, "r"),
                               _ptr(q, n, _F64, "q", allow_none=model != FV_BSM),
                               _ptr(flag, n, _I8, "flag"), n, _ptr(out_sigma, n, _F64, "out_sigma"),
                               _ptr(status, n, _U8, "status"), _stream(stream)), "fv_implied_vol")
    return out_sigma, status


def fv_workspace_size(solver, n):
    return int(_lib.fv_workspace_size(solver, n))


def fv_implied_vol_ws(model, solver, price, S_or_F, K, T, r, q, flag, workspace, out_sigma=None,
                      status=None, stream=None):
    n = price.numel()
    out_sigma, status = _iv_outputs(price, out_sigma, status)
    if workspace is None:
        wp, wb = None, 0
    else:
        if not workspace.is_cuda or not workspace.is_contiguous():
            raise TypeError("workspace must be a contiguous CUDA tensor")
        wp, wb = ctypes.c_void_p(workspace.data_ptr()), workspace.numel() * workspace.element_size()
    _check(_lib.fv_implied_vol_ws(model, solver, _ptr(price, n, _F64, "price"),
                                  _ptr(S_or_F, n, _F64, "S_or_F"), _ptr(K, n, _F64, "K"),
                                  _ptr(T, n, _F64, "T"), _ptr(r, n, _F64, "r"),
                                  _ptr(q, n, _F64, "q", allow_none=model != FV_BSM),
                                  _ptr(flag, n, _I8, "flag"), n,
                                  _ptr(out_sigma, n, _F64, "out_sigma"),
                                  _ptr(status, n, _U8, "status"), wp, wb, _stream(stream)),
           "fv_implied_vol_ws")
    return out_sigma, status


FV_NOALLOC_MAX_QUOTES = 262144


def fv_implied_vol_halley_noalloc(model, price, S_or_F, K, T, r, q, flag, out_sigma=None,
                                  status=None, stream=None):
    """Halley implied volatility using the library's built-in scratch array
    instead of any device allocation (at most FV_NOALLOC_MAX_QUOTES quotes;
    calls must not overlap on the GPU)."""
    n = price.numel()
    out_sigma, status = _iv_outputs(price, out_sigma, status)
    _check(_lib.fv_implied_vol_halley_noalloc(
        model, _ptr(price, n, _F64, "price"), _ptr(S_or_F, n, _F64, "S_or_F"),
        _ptr(K, n, _F64, "K"), _ptr(T, n, _F64, "T"), _ptr(r, n, _F64, "r"),
        _ptr(q, n, _F64, "q", allow_none=model != FV_BSM), _ptr(flag, n, _I8, "flag"), n,
        _ptr(out_sigma, n, _F64, "out_sigma"), _ptr(status, n, _U8, "status"), _stream(stream)),
        "fv_implied_vol_halley_noalloc")
    return out_sigma, status


def fv_implied_vol_ex(model, solver, precision, price, S_or_F, K, T, r, q, flag, out_sigma=None,
                      status=None, stream=None):
    n = price.numel()
    if price.dtype == torch.float32:
        dt, dts = FV_DTYPE_F32, _F32
    else:
        dt, dts = FV_DTYPE_F64, _F64
    out_sigma, status = _iv_outputs(price, out_sigma, status)
    _check(_lib.fv_implied_vol_ex(model, solver, precision, dt, _ptr(price, n, dts, "price"),
                                  _ptr(S_or_F, n, dts, "S_or_F"), _ptr(K, n, dts, "K"),
                                  _ptr(T, n, dts, "T"), _ptr(r, n, dts, "r"),
                                  _ptr(q, n, dts, "q", allow_none=model != FV_BSM),
                                  _ptr(flag, n, _I8, "flag"), n,
                                  _ptr(out_sigma, n, _F64, "out_sigma"),
                                  _ptr(status, n, _U8, "status"), _stream(stream)),
           "fv_implied_vol_ex")
    return out_sigma, status


def fv_implied_vol_strided(model, solver, precision, price, S_or_F, K, T, r, q, flag,
                           out_sigma=None, status=None, stream=None):
    """Implied volatility where any input may hold one element (broadcast to
    every quote, stride 0) or n elements (stride 1)."""
    ins = [price, S_or_F, K, T, r, q, flag]
    n = max(t.numel() for t in ins if t is not None)
    f32 = price.dtype == torch.float32
    dts = _F32 if f32 else _F64
    strides = (ctypes.c_int64 * 7)()
    ptrs = []
    for k, (t, name) in enumerate(zip(ins, ("price", "S_or_F", "K", "T", "r", "q", "flag"))):
        if t is None:
            if name != "q" or model == FV_BSM:
                raise ValueError("%s is required" % name)
            ptrs.append(None)
            strides[k] = 0
            continue
        m = t.numel()
        if m not in (1, n):
            raise ValueError("%s has %d elements: expected 1 or %d" % (name, m, n))
        ptrs.append(_ptr(t, m, _I8 if name == "flag" else dts, name))
        strides[k] = 0 if (m == 1 and n != 1) else 1
    ref = price if price.numel() == n else S_or_F
    out_sigma = torch.empty(n, dtype=torch.float64, device=ref.device) if out_sigma is None else out_sigma
    status = torch.empty(n, dtype=torch.uint8, device=ref.device) if status is None else status
    _check(_lib.fv_implied_vol_strided(model, solver, precision, FV_DTYPE_F32 if f32 else FV_DTYPE_F64,
                                       *ptrs, strides, n, _ptr(out_sigma, n, _F64, "out_sigma"),
                                       _ptr(status, n, _U8, "status"), _stream(stream)),
           "fv_implied_vol_strided")
    return out_sigma, status


def fv_greeks(model, flag, S_or_F, K, T, r, q, sigma, outputs=("delta", "gamma", "vega", "theta",
                                                               "rho"), stream=None):
    """Returns a dict name -> tensor for the requested Greeks."""
    n = S_or_F.numel()
    res = {k: _like(S_or_F, torch.float64) for k in outputs}
    ptrs = [ctypes.c_void_p(res[k].data_ptr()) if k in res else None
            for k in ("delta", "gamma", "vega", "theta", "rho")]
    _check(_lib.fv_greeks(model, _ptr(flag, n, _I8, "flag"), _ptr(S_or_F, n, _F64, "S_or_F"),
                          _ptr(K, n, _F64, "K"), _ptr(T, n, _F64, "T"), _ptr(r, n, _F64, "r"),
                          _ptr(q, n, _F64, "q", allow_none=model != FV_BSM),
                          _ptr(sigma, n, _F64, "sigma"), n, *ptrs, _stream(stream)), "fv_greeks")
    return res


def fv_iv_adjoint(model, price, S_or_F, K, T, r, q, flag, sigma, status, grad_sigma,
                  outputs=("P", "S", "K", "T", "r", "q"), stream=None):
    """Returns a dict input name -> grad_sigma * d sigma / d input."""
    n = S_or_F.numel()
    res = {k: _like(S_or_F, torch.float64) for k in outputs}
    ptrs = [ctypes.c_void_p(res[k].data_ptr()) if k in res else None
            for k in ("P", "S", "K", "T", "r", "q")]
    _check(_lib.fv_iv_adjoint(model, _ptr(price, n, _F64, "price", allow_none=model != FV_BLACK76),
                              _ptr(S_or_F, n, _F64, "S_or_F"), _ptr(K, n, _F64, "K"),
                              _ptr(T, n, _F64, "T"), _ptr(r, n, _F64, "r"),
                              _ptr(q, n, _F64, "q", allow_none=model != FV_BSM),
                              _ptr(flag, n, _I8, "flag"), _ptr(sigma, n, _F64, "sigma"),
                              _ptr(status, n, _U8, "status"),
                              _ptr(grad_sigma, n, _F64, "grad_sigma"), n, *ptrs, _stream(stream)),
           "fv_iv_adjoint")
    return res


def fv_normalised_black(x, s, theta, out=None, stream=None):
    n = x.numel()
    out = _like(x, torch.float64) if out is None else out
    _check(_lib.fv_normalised_black(_ptr(x, n, _F64, "x"), _ptr(s, n, _F64, "s"),
                                    _ptr(theta, n, _I8, "theta"), n, _ptr(out, n, _F64, "out"),
                                    _stream(stream)), "fv_normalised_black")
    return out


FV_MATH_ERFCX, FV_MATH_LOG, FV_MATH_EXP, FV_MATH_EXPM1, FV_MATH_LOG1P, FV_MATH_ERFCX_SQRT2 = 0, 1, 2, 3, 4, 5


def fv_math(which, z, out=None, stream=None):
    n = z.numel()
    out = _like(z, torch.float64) if out is None else out
    _check(_lib.fv_math(which, _ptr(z, n, _F64, "z"), n, _ptr(out, n, _F64, "out"),
                        _stream(stream)), "fv_math")
    return out


class fv_chains_plan:
    """A plan over many option chains (one persistent launch captured in a CUDA graph).

    chains: list of dicts with device tensors price, K, flag, sigma, status and
    scalars S_or_F, T, r (and q for BSM).  The tensors must outlive the plan.
    """

    def __init__(self, model, chains, solver=FV_LBR, autotune=True, stream=None):
        arr = (fv_chain * max(1, len(chains)))()
        self._keep = chains
        for i, c in enumerate(chains):
            n = c["price"].numel()
            arr[i].price = c["price"].data_ptr() if n else None
            arr[i].K = c["K"].data_ptr() if n else None
            arr[i].flag = c["flag"].data_ptr() if n else None
            arr[i].sigma = c["sigma"].data_ptr() if n else None
            arr[i].status = c["status"].data_ptr() if n else None
            arr[i].n = n
            arr[i].S_or_F = float(c["S_or_F"])
            arr[i].T = float(c["T"])
            arr[i].r = float(c["r"])
            arr[i].q = float(c.get("q", 0.0))
        h = ctypes.c_void_p()
        _check(_lib.fv_chains_plan_create(model, solver, arr, len(chains), int(bool(autotune)),
                                          _stream(stream), ctypes.byref(h)), "fv_chains_plan_create")
        self._h = h

    def run(self, stream=None):
        _check(_lib.fv_implied_vol_chains(self._h, _stream(stream)), "fv_implied_vol_chains")

    def run_direct(self, stream=None):
        _check(_lib.fv_implied_vol_chains_direct(self._h, _stream(stream)),
               "fv_implied_vol_chains_direct")

    def info(self):
        b, q, g = _I(), _I(), _I()
        t, n = _N(), _N()
        _check(_lib.fv_chains_plan_info(self._h, ctypes.byref(b), ctypes.byref(q), ctypes.byref(g),
                                        ctypes.byref(t), ctypes.byref(n)), "fv_chains_plan_info")
        return dict(block=b.value, quotes_per_thread=q.value, grid=g.value, tiles=t.value,
                    quotes=n.value)

    def tuning(self):
        """How the launch shape was chosen: blocks_per_sm, source ("default",
        "timed" or "cached"), candidates timed, best_ms and the tuning key."""
        b, src, c = _I(), _I(), _I()
        ms = ctypes.c_double()
        key = ctypes.create_string_buffer(512)
        _check(_lib.fv_chains_plan_tuning(self._h, ctypes.byref(b), ctypes.byref(src), ctypes.byref(c),
                                          ctypes.byref(ms), key, 512), "fv_chains_plan_tuning")
        return dict(blocks_per_sm=b.value, source=("default", "timed", "cached")[src.value],
                    candidates=c.value, best_ms=ms.value, key=key.value.decode())

    def destroy(self):
        if getattr(self, "_h", None):
            _lib.fv_chains_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def fv_autotune_cache_get(path, key):
    """The tuning-cache entry for key: dict(block, quotes_per_thread,
    blocks_per_sm, ms), or None when the file or the entry is absent."""
    b, q, s = _I(), _I(), _I()
    ms = ctypes.c_double()
    _check(_lib.fv_autotune_cache_get(os.fsencode(path), key.encode(), ctypes.byref(b), ctypes.byref(q),
                                      ctypes.byref(s), ctypes.byref(ms)), "fv_autotune_cache_get")
    if b.value == 0:
        return None
    return dict(block=b.value, quotes_per_thread=q.value, blocks_per_sm=s.value, ms=ms.value)


def fv_autotune_cache_put(path, key, block, quotes_per_thread, blocks_per_sm, ms=0.0):
    _check(_lib.fv_autotune_cache_put(os.fsencode(path), key.encode(), int(block),
                                      int(quotes_per_thread), int(blocks_per_sm), float(ms)),
           "fv_autotune_cache_put")


def _host_ptr(t, n, dtypes, name, allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise ValueError("%s is required" % name)
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError("%s must be a host (CPU) tensor" % name)
    if t.dtype not in dtypes or not t.is_contiguous() or t.numel() != n:
        raise ValueError("%s must be a contiguous %s tensor with %d elements" % (name, dtypes, n))
    return ctypes.c_void_p(t.data_ptr())


class fv_stream_plan:
    """Host-resident batches (see fv_implied_vol_host).  With pinned host
    tensors (tensor.pin_memory()) the solver reads and writes them in place
    over the CPU-GPU link (FV_TRANSFER_DIRECT); otherwise the plan's device
    staging and two streams copy them in chunks overlapped with the solve
    (FV_TRANSFER_STAGED).  set_transfer() forces one of the two."""

    def __init__(self, chunk_quotes=1 << 21):
        h = ctypes.c_void_p()
        _check(_lib.fv_stream_plan_create(int(chunk_quotes), ctypes.byref(h)), "fv_stream_plan_create")
        self._h = h

    def set_transfer(self, mode):
        _check(_lib.fv_stream_plan_set_transfer(self._h, int(mode)), "fv_stream_plan_set_transfer")

    @property
    def last_transfer(self):
        """The mode the last call took (FV_TRANSFER_AUTO before the first)."""
        m = _I()
        _check(_lib.fv_stream_plan_last_transfer(self._h, ctypes.byref(m)),
               "fv_stream_plan_last_transfer")
        return m.value

    def implied_vol(self, model, solver, precision, price, S_or_F, K, T, r, q, flag, out_sigma=None,
                    status=None, stream=None):
        n = price.numel()
        f32 = price.dtype == torch.float32
        dts = _F32 if f32 else _F64
        if out_sigma is None:
            out_sigma = torch.empty(n, dtype=torch.float64, pin_memory=True)
        if status is None:
            status = torch.empty(n, dtype=torch.uint8, pin_memory=True)
        _check(_lib.fv_implied_vol_host(
            self._h, model, solver, precision, FV_DTYPE_F32 if f32 else FV_DTYPE_F64,
            _host_ptr(price, n, dts, "price"), _host_ptr(S_or_F, n, dts, "S_or_F"),
            _host_ptr(K, n, dts, "K"), _host_ptr(T, n, dts, "T"), _host_ptr(r, n, dts, "r"),
            _host_ptr(q, n, dts, "q", allow_none=model != FV_BSM), _host_ptr(flag, n, _I8, "flag"), n,
            _host_ptr(out_sigma, n, _F64, "out_sigma"), _host_ptr(status, n, _U8, "status"),
            _stream(stream)), "fv_implied_vol_host")
        return out_sigma, status

    def destroy(self):
        if getattr(self, "_h", None):
            _lib.fv_stream_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def fv_stream_plan_create(chunk_quotes=1 << 21):
    return fv_stream_plan(chunk_quotes)


def fv_implied_vol_host(plan, model, solver, precision, price, S_or_F, K, T, r, q, flag,
                        out_sigma=None, status=None, stream=None):
    return plan.implied_vol(model, solver, precision, price, S_or_F, K, T, r, q, flag, out_sigma,
                            status, stream)


def fv_stream_plan_destroy(plan):
    plan.destroy()


def fv_chains_plan_create(model, chains, solver=FV_LBR, autotune=True, stream=None):
    return fv_chains_plan(model, chains, solver, autotune, stream)


def fv_implied_vol_chains(plan, stream=None):
    plan.run(stream)


def fv_chains_plan_destroy(plan):
    plan.destroy()


class ImpliedVol(torch.autograd.Function):
    """sigma = IV(P, S|F, K, T, r, q) with the library's adjoint in backward.

    forward runs fv_implied_vol (FP64 LBR); backward runs fv_iv_adjoint at the
    converged sigma (implicit-function theorem, no stored iterations).
    """

    @staticmethod
    def forward(ctx, price, S_or_F, K, T, r, q, flag, model=FV_BSM, solver=FV_LBR):
        sigma, status = fv_implied_vol(model, solver, price, S_or_F, K, T, r, q, flag)
        ctx.model = model
        ctx.has_q = q is not None
        ctx.save_for_backward(price, S_or_F, K, T, r, q if q is not None else price, flag, sigma,
                              status)
        ctx.mark_non_differentiable(status)
        return sigma, status

    @staticmethod
    def backward(ctx, grad_sigma, grad_status):
        price, S_or_F, K, T, r, q, flag, sigma, status = ctx.saved_tensors
        q = q if ctx.has_q else None
        g = fv_iv_adjoint(ctx.model, price, S_or_F, K, T, r, q, flag, sigma, status,
                          grad_sigma.contiguous())
        return (g["P"], g["S"], g["K"], g["T"], g["r"], g["q"] if ctx.has_q else None, None, None,
                None)


def implied_volatility_autograd(price, S_or_F, K, T, r, q, flag, model=FV_BSM, solver=FV_LBR):
    """Differentiable implied volatility (returns sigma; status is discarded)."""
    return ImpliedVol.apply(price, S_or_F, K, T, r, q, flag, model, solver)[0]
