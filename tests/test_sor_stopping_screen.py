"""The red-black SOR's stopping test asks, per cell, whether fl(|d| / |Phi_new|) >= tol (d = Phi_new - Phi_old,
the relative change of Sec. 2.3's iteration). The GPU kernel takes that decision mostly without a division:
from the exponents alone when the ratio is at least a factor of two away from tol, else from an FP32 estimate
of the leading 20 mantissa bits, dividing in FP64 only when the estimate is within 2^-14 of tol. These CPU
tests replay that screen on the host, with the FP32 fast division taken anywhere inside its documented
2-ulp error bound (both extremes and exact), and check that every branch returns the plain decision."""
import math
import random
import struct

import numpy as np

F32_DIV_REL = 2.0 ** -22  # 2 ulps of an FP32 result, relative


def _hi(x):
    return struct.unpack("<q", struct.pack("<d", x))[0] >> 32


def _f32_bits(b):
    return np.frombuffer(struct.pack("<I", b), dtype=np.float32)[0]


def _screen(d, nw, tol, delta):
    """The kernel's decision for a nonzero d, with the fast FP32 division off by the relative amount delta."""
    plain = abs(d) / abs(nw) >= tol
    m, e2 = math.frexp(tol)
    tol_exp, tol_mant = e2 - 1, np.float32(2.0 * m)
    hd, hn = _hi(d), _hi(nw)
    ed, en = (hd >> 20) & 0x7FF, (hn >> 20) & 0x7FF
    if not (math.isfinite(tol) and tol > 0 and tol >= 2.2250738585072014e-308) or ed in (0, 0x7FF) or en in (0, 0x7FF):
        return plain, "divide"
    k = ed - en - tol_exp
    if k >= 2:
        return True, "exponent"
    if k <= -2:
        return False, "exponent"
    fd = _f32_bits(0x3F800000 | ((hd & 0xFFFFF) << 3))
    fn = _f32_bits(0x3F800000 | ((hn & 0xFFFFF) << 3))
    den = np.float32(fn * tol_mant)
    q = np.float32(float(fd) / float(den) * (1.0 + delta))
    est = np.float32(q * np.float32(1.0 if k == 0 else (2.0 if k > 0 else 0.5)))
    if est >= np.float32(1.0 + 2.0 ** -14):
        return True, "estimate"
    if est > np.float32(1.0 - 2.0 ** -14):
        return plain, "divide"
    return False, "estimate"


def _check(d, nw, tol, seen):
    want = abs(d) / abs(nw) >= tol
    for delta in (-F32_DIV_REL, 0.0, F32_DIV_REL):
        got, how = _screen(d, nw, tol, delta)
        seen.add(how)
        assert got == want, (d.hex(), nw.hex(), tol.hex(), delta, how)


def test_random_ratios_over_wide_ranges():
    rnd = random.Random(20150730)
    seen = set()
    for _ in range(40000):
        tol = math.ldexp(rnd.uniform(1, 2), rnd.randint(-60, -3))
        nw = math.ldexp(rnd.uniform(1, 2), rnd.randint(-200, 200)) * rnd.choice((-1, 1))
        d = abs(nw) * tol * math.ldexp(rnd.uniform(0.5, 2), rnd.randint(-3, 3)) * rnd.choice((-1, 1))
        _check(d, nw, tol, seen)
    assert {"exponent", "estimate"} <= seen  # random ratios almost never fall within 2^-14 of tol


def test_ratios_next_to_tol():
    """|d| / |nw| a few ulps either side of tol, where only the division can decide, and ratios on both sides
    of the estimate's 2^-14 screen."""
    rnd = random.Random(7)
    seen = set()
    for _ in range(20000):
        tol = rnd.choice((1e-8, 2.0 ** -30, 3.7e-9, 1e-6, math.ldexp(rnd.uniform(1, 2), rnd.randint(-50, -5))))
        nw = math.ldexp(rnd.uniform(1, 2), rnd.randint(-60, 60))
        for rel in (rnd.randint(-4, 4) * 2.0 ** -52, rnd.choice((-1, 1)) * 2.0 ** -14 * rnd.uniform(0.9, 1.1),
                    rnd.choice((-1, 1)) * rnd.uniform(2.0 ** -14, 2.0 ** -8)):
            d = nw * tol * (1.0 + rel)
            _check(d, nw, tol, seen)
            _check(-d, -nw, tol, seen)
    assert {"estimate", "divide"} <= seen
