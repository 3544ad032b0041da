"""The Planck-integral polynomials of the CUDA library (csrc/planck_table.h,
written by csrc/gen_planck_table.py) against the oracle's series evaluation of
P(x) and Q(x), on the CPU.  The polynomials are evaluated here the way the
device evaluates them (segment from the binary exponent and two leading
mantissa bits, Horner in u; the device's fused multiply-adds only make its
evaluation more accurate than this one)."""
import math
import os
import re
import struct

import numpy as np
import pytest

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "..", "paper_2407_18304_gb300", "csrc", "planck_table.h")
K = 15.0 / math.pi ** 4


def _table():
    txt = open(HEADER).read()
    ints = {k: int(v) for k, v in re.findall(r"constexpr int (k\w+) = (-?\d+);", txt)}

    def arr(name):
        body = re.search(name + r"[^=]*= \{(.*?)\};", txt, re.S).group(1)
        return [float.fromhex(t) for t in re.findall(r"-?0x[0-9a-fp.+-]+", body)]

    deg, nseg = ints["kDeg"], ints["kSeg"]
    coef = np.array(arr("kCoef")).reshape(deg + 1, nseg)
    return ints, np.array(arr("kCentre")), np.array(arr("kInvHalf")), coef


def _eval(x, ints, cen, ih, coef):
    """P(x) (x < 2) or Q(x) (x >= 2) as the device computes it."""
    hi = struct.unpack("<q", struct.pack("<d", x))[0] >> 32
    e = ((hi >> 20) & 0x7FF) - 1023
    s = 1 + (e - ints["kEMin"]) * ints["kSub"] + ((hi >> 18) & 3)
    s = 0 if e < ints["kEMin"] else (ints["kSeg"] - 1 if e > ints["kEMax"] else s)
    u = 0.0 if e > ints["kEMax"] else (x - cen[s]) * ih[s]
    p = coef[ints["kDeg"], s]
    for k in range(ints["kDeg"] - 1, -1, -1):
        p = p * u + coef[k, s]
    x3 = x * x * x
    return K * x3 * p if x < 2.0 else K * x3 * p * math.exp(-x)


def test_table_matches_the_oracle_series():
    ints, cen, ih, coef = _table()
    xs = np.concatenate([np.logspace(-6, math.log10(700.0), 3001),
                         [2.0 ** e for e in range(-9, 10)], [1.999999999999, 2.0, 2.0000000001]])
    worst_p = worst_q = 0.0
    for x in xs:
        x = float(x)
        v = _eval(x, ints, cen, ih, coef)
        if x < 2.0:
            ref = O.planck_P(x)
            worst_p = max(worst_p, abs(v - ref) / ref)
        else:
            ref = O.planck_Q(x)
            if ref > 0.0:
                worst_q = max(worst_q, abs(v - ref) / ref)
    print(f"worst relative error: P {worst_p:.2e}, Q {worst_q:.2e}")
    # the device evaluates with fused multiply-adds; the oracle's series are
    # themselves accurate to a few ulp
    assert worst_p < 1e-15 and worst_q < 1e-15


def test_segments_tile_the_line():
    ints, cen, ih, coef = _table()
    # segment s covers [c - w, c + w]; consecutive segments touch
    lo = cen - 1.0 / ih
    hi = cen + 1.0 / ih
    assert lo[0] == 0.0 and hi[0] == 2.0 ** ints["kEMin"]
    assert np.all(np.abs(hi[:-1] - lo[1:]) <= 1e-15 * hi[:-1])
    assert hi[-1] == 2.0 ** (ints["kEMax"] + 1)


def test_fp32_truncation_is_below_fp32_resolution():
    """The FP32 passes use the same polynomials cut to degree 7 in FP32."""
    ints, cen, ih, coef = _table()
    f32 = np.float32
    worst = 0.0
    for x in np.logspace(-4, math.log10(80.0), 2001):
        xf = f32(x)
        hi = struct.unpack("<i", struct.pack("<f", xf))[0]
        e = ((hi >> 23) & 0xFF) - 127
        s = 1 + (e - ints["kEMin"]) * ints["kSub"] + ((hi >> 21) & 3)
        s = 0 if e < ints["kEMin"] else (ints["kSeg"] - 1 if e > ints["kEMax"] else s)
        u = (xf - f32(cen[s])) * f32(ih[s])
        p = f32(coef[7, s])
        for k in range(6, -1, -1):
            p = f32(p * u + f32(coef[k, s]))
        x = float(xf)
        x3 = x * x * x
        v = K * x3 * float(p) if x < 2.0 else K * x3 * float(p) * math.exp(-x)
        ref = O.planck_P(x) if x < 2.0 else O.planck_Q(x)
        worst = max(worst, abs(v - ref) / ref)
    print(f"worst FP32 relative error {worst:.2e}")
    assert worst < 1e-6


def test_table_is_what_its_generator_writes(tmp_path):
    """The committed polynomials are exactly the generator's output (50-digit
    mpmath fits, each segment checked at 400 points): nothing in the header
    was edited by hand.  About half a minute."""
    import importlib.util

    pytest.importorskip("mpmath")
    gen = os.path.join(os.path.dirname(HEADER), "gen_planck_table.py")
    spec = importlib.util.spec_from_file_location("gen_planck_table", gen)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    out = tmp_path / "planck_table.h"
    mod.main(str(out))
    assert out.read_bytes() == open(HEADER, "rb").read()
