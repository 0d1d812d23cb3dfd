"""The FP64 erfcx table of the CUDA kernels, checked on the CPU.

The kernels evaluate erfcx(z) = exp(z^2) erfc(z) on 0 <= z < 128 from
piecewise Chebyshev interpolants (csrc/fv_erfcx_table.h, written by
csrc/gen_erfcx_table.py).  Here the committed table is (1) what the generator
writes, and (2) within one ulp of mpmath's erfcx when evaluated the way the
kernel does (piece located from the bits of z, Horner with exactly rounded
fused multiply-adds), on points the generator never looked at.
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
HEADER = os.path.join(CSRC, "fv_erfcx_table.h")


def _gen():
    spec = importlib.util.spec_from_file_location("gen_erfcx_table",
                                                  os.path.join(CSRC, "gen_erfcx_table.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _table():
    src = open(HEADER).read()
    stride = int(re.search(r"#define FV_ERFCX_STRIDE (\d+)", src).group(1))
    body = src[src.index("{") + 1:src.index("};")]
    vals = [float(v) for v in body.replace("\n", " ").split(",") if v.strip()]
    return np.array(vals).reshape(-1, stride)


def _piece(z):
    if z < 0.5:
        return int(z * 8.0)
    hi = struct.unpack("<q", struct.pack("<d", z))[0] >> 32
    return 4 + (((hi >> 20) - 1022) << 3) + ((hi >> 17) & 7)


def _fma(x, y, z):
    return float(mp.mpf(x) * mp.mpf(y) + mp.mpf(z))


def _eval(tab, z):
    row = tab[_piece(z)]
    v = z - row[0]
    p = row[11]
    for j in range(10, 0, -1):
        p = _fma(p, v, row[j])
    return p


def test_committed_table_is_the_generators_output(tmp_path):
    out = str(tmp_path / "table.h")
    _gen().main(out=out, samples=4)
    assert open(out).read() == open(HEADER).read()


def test_table_within_one_ulp_of_erfcx():
    mp.mp.dps = 40
    tab = _table()
    g = np.random.default_rng(5)
    # random points in every piece, the piece edges and their neighbours
    edges = [k / 8 for k in range(5)] + [2.0 ** e * (1 + j / 8) for e in range(-1, 7)
                                         for j in range(8)]
    z = np.concatenate([g.uniform(0, 0.5, 300), np.exp(g.uniform(np.log(0.5), np.log(128), 1200)),
                        edges, np.nextafter(edges, 0), np.nextafter(edges, 200), [0.0, 5e-324]])
    z = z[(z >= 0) & (z < 128)]
    worst = 0.0
    for zi in z:
        ref = mp.exp(mp.mpf(zi) ** 2) * mp.erfc(mp.mpf(zi))
        worst = max(worst, abs(float((_eval(tab, float(zi)) - ref) / ref)))
    assert worst <= 2.0 ** -52, worst
