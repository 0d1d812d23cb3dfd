"""fv_implied_vol_halley_noalloc: the Halley entry point for callers that may not
allocate device memory (its fallback list lives in a scratch array built into
the library instead of a cudaMalloc'd workspace).

Checked through the C ABI against fv_implied_vol (Halley) on two calls in a
row with different inputs, both sending quotes to the fallback and in
different numbers, so the second call must start from a cleared scratch
counter and must not reuse the first call's list.  This file is collected
last on purpose.
"""
import ctypes

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2604_27210_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _inputs(torch, dev, seed, n_maturities):
    # a strike x maturity grid: wing quotes make the fallback run
    w = wl.fill_prices(wl.bsm_grid(512, n_maturities, seed=seed), orc.price)
    t = {k: torch.tensor(np.ascontiguousarray(w[k]), device=dev)
         for k in ("P", "S_or_F", "K", "T", "r", "q", "flag")}
    return w, t


def _fallback_count(fv, torch, t):
    """Quotes the Halley sweeps hand to the fallback for these inputs: the same
    kernels run through fv_implied_vol_ws with a workspace of our own, whose
    first four bytes are the compacted list's length after the call."""
    n = t["P"].numel()
    ws = torch.zeros(fv.fv_workspace_size(fv.FV_HALLEY, n), dtype=torch.uint8, device=t["P"].device)
    fv.fv_implied_vol_ws(fv.FV_BSM, fv.FV_HALLEY, t["P"], t["S_or_F"], t["K"], t["T"], t["r"],
                         t["q"], t["flag"], ws)
    torch.cuda.synchronize()
    return int(ws[:4].cpu().numpy().view(np.uint32)[0])


def _call(lib, t, n, sigma, status, stream):
    p = lambda x: ctypes.c_void_p(x.data_ptr())
    return lib.fv_implied_vol_halley_noalloc(
        2, p(t["P"]), p(t["S_or_F"]), p(t["K"]), p(t["T"]), p(t["r"]), p(t["q"]), p(t["flag"]),
        ctypes.c_int64(n), p(sigma), p(status), ctypes.c_void_p(stream))


def test_noalloc_matches_halley_on_two_calls():
    import torch
    from paper_2604_27210_gb300 import fv

    dev = torch.device("cuda:0")
    lib = fv.library()
    stream = torch.cuda.current_stream().cuda_stream
    counts = []
    for seed, n_m in ((1, 200), (5, 150)):  # two calls in a row, different quotes
        w, t = _inputs(torch, dev, seed, n_m)
        n = t["P"].numel()
        assert n <= fv.FV_NOALLOC_MAX_QUOTES
        counts.append(_fallback_count(fv, torch, t))
        assert counts[-1] > 0, "the fallback must run on this call"
        s_ref, st_ref = fv.fv_implied_vol(fv.FV_BSM, fv.FV_HALLEY, t["P"], t["S_or_F"], t["K"],
                                          t["T"], t["r"], t["q"], t["flag"])
        sigma = torch.full((n,), -1.0, dtype=torch.float64, device=dev)
        status = torch.full((n,), 99, dtype=torch.uint8, device=dev)
        rc = _call(lib, t, n, sigma, status, stream)
        assert rc == fv.FV_SUCCESS, lib.fv_last_error()
        torch.cuda.synchronize()
        st_a, st_b = status.cpu().numpy(), st_ref.cpu().numpy()
        s_a, s_b = sigma.cpu().numpy(), s_ref.cpu().numpy()
        assert np.array_equal(st_a, st_b)
        assert np.array_equal(np.isnan(s_a), np.isnan(s_b))
        ok = ~np.isnan(s_b) & (s_b > 0)
        # the same per-quote arithmetic in both arrangements (compacted list
        # here, per-tile lists in fv_implied_vol): only rounding may differ
        assert np.all(np.abs(s_a[ok] - s_b[ok]) <= 1e-12 * s_b[ok])
        assert np.all(s_a[~np.isnan(s_b) & (s_b == 0)] == 0)
        # most quotes are solved; the grid's wing quotes go through the fallback
        assert (st_b == orc.OK).sum() > 0.5 * n
    assert counts[0] != counts[1], counts


def test_noalloc_rejects_oversized_batches():
    import torch
    from paper_2604_27210_gb300 import fv

    lib = fv.library()
    dev = torch.device("cuda:0")
    x = torch.ones(4, dtype=torch.float64, device=dev)
    p = ctypes.c_void_p(x.data_ptr())
    rc = lib.fv_implied_vol_halley_noalloc(2, p, p, p, p, p, p, p,
                                           ctypes.c_int64(fv.FV_NOALLOC_MAX_QUOTES + 1), p, p, None)
    assert rc == fv.FV_ERR_ARG
    assert b"FV_NOALLOC_MAX_QUOTES" in lib.fv_last_error()
    torch.cuda.synchronize()
