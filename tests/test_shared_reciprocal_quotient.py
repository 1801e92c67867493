"""The FP64 WENO5 weights divide three values by their common sum s through one reciprocal y = RN(1/s):
q = RN(a y), r = RN(a - q s) (a fused multiply-add), q' = RN(q + r y). These CPU tests check, in exact
rational arithmetic (CPython's integer true division rounds correctly, so a fused multiply-add is the exact
value rounded once), that q' is the IEEE quotient RN(a / s) for normal operands, so that the FP64 stage
kernel stays bitwise equal to a plain evaluation with true divisions.

Why it holds. Scale a, b into [1, 2) and let u = 2^-53. If a >= b the quotient lies in [1, 2), q is within
one ulp and Markstein's theorem (IBM J. Res. Dev. 34, 1990) gives RN(a / b). If a < b, q can be up to
1.5 ulps away (y's error a/2 ulp plus q's rounding), so r may be rounded; the corrected value then lies
within 2u^2/b + 0.75 b u^2 + u^3 <= 2.75 u^2 + u^3 of a / b, while a quotient whose q is not faithful sits
more than (k + 1) u^2 from every rounding midpoint, for b = 2 - 2ku. That leaves only k = 1 (b the largest
double below 2), which the exhaustive corner test covers."""
import math
import random
from fractions import Fraction as Fr


def _fma(x, y, z):
    return float(Fr(x) * Fr(y) + Fr(z))


def _shared(a, b, y):
    q = a * y
    r = _fma(-q, b, a)
    return _fma(r, y, q)


def test_weight_like_quotients():
    rnd = random.Random(20150730)
    for _ in range(20000):
        e = [10 ** rnd.uniform(-6, 9) * rnd.uniform(1, 2) for _ in range(3)]
        w = [d / (x * x) for d, x in zip((0.1, 0.6, 0.3), e)]
        s = (w[0] + w[1]) + w[2]
        y = 1.0 / s
        for a in w:
            assert _shared(a, s, y) == a / s


def test_unfaithful_first_quotients_next_to_midpoints():
    """b = (2^53 - k) 2^-52 with k odd (1/b a near tie, so y is off by almost half an ulp) and a chosen so
    that a / b lies within |d| 2^-106 / b of a rounding midpoint: many first quotients are more than an ulp
    off, and the corrected one must still be RN(a / b)."""
    two54, unfaithful, n = 1 << 54, 0, 0
    for k in range(1, 600, 2):
        B = (1 << 53) - k
        b = B / 2.0 ** 52
        y = 1.0 / b
        inv = pow(two54, -1, B)
        for d in range(-12, 13):
            A = (d * inv) % B
            if d == 0 or not (1 << 52) <= A < B:
                continue
            a = A / 2.0 ** 52
            exact = Fr(a) / Fr(b)
            unfaithful += abs(Fr(a * y) - exact) >= Fr(math.ulp(float(exact)))
            n += 1
            assert _shared(a, b, y) == a / b
    assert unfaithful > n // 10  # the construction does reach the case Markstein's theorem leaves out


def test_corner_exhaustively():
    """Every pair a < b among the 400 largest doubles below 2, and the same pairs scaled by powers of two."""
    top = 1 << 53
    for B in range(top - 400, top):
        b = B / 2.0 ** 52
        y = 1.0 / b
        for A in range(top - 400, B):
            a = A / 2.0 ** 52
            assert _shared(a, b, y) == a / b
    for sa, sb in ((2.0 ** -30, 2.0 ** 12), (2.0 ** 40, 2.0 ** -7)):
        b = (top - 1) / 2.0 ** 52 * sb
        a = (top - 2) / 2.0 ** 52 * sa
        assert _shared(a, b, 1.0 / b) == a / b
