"""Accuracy of the Schwinger sum's cosine (Sec. 2.2: Delta(t) sums w_n cos(t p_n)),
checked on the CPU by an emulation of the kernel's arithmetic against 40-digit values.

The kernel reduces x by Cody-Waite with pi/2 in two FP64 parts (k = nearest integer to
2x/pi by the 1.5 2^52 shifter; below |x| = 2^18, k = the FP32 product of the leading 24
bits of x and 2/pi rounded to an integer, which can miss the nearest integer by one
near a half-integer; r = x - k P1 - k P2 by FMA).  It then takes
cos x = +-cos r or -+sin r by the quadrant.  The leading Taylor terms 1 - r^2/2 and
r - r^3/6 are one FP64 FMA, and the tails r^4 (1/4! - ...) and r^5 (1/5! - ...) are
in double-float.  The emulation repeats those operations: FP64 ones with one rounding,
FP32 ones in numpy float32.  The test pins the kernel's claim that lead + tail is
within a few units of 2^-53 of cos x for |x| < 2^49.  A planted mistake (pi/2 in one
part) fails.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from df_emulation import _dmul, _fma64, _muladd, _split

mpmath = pytest.importorskip("mpmath")

P1 = 1.5707963267948966        # pi/2 rounded to FP64
P2 = 6.123233995736766e-17     # pi/2 - P1 rounded to FP64
TWO_OVER_PI = 0.6366197723675814
SHIFTER = 6755399441055744.0   # 1.5 2^52


def _tail_coefficients():
    c, s = [], []
    fc, fs = 24.0, 120.0  # (2k + 4)!, (2k + 5)!
    for k in range(8):
        sg = -1.0 if k & 1 else 1.0
        c.append(_split(sg / fc))
        s.append(_split(sg / fs))
        fc *= (2 * k + 5) * (2 * k + 6)
        fs *= (2 * k + 6) * (2 * k + 7)
    return c, s


_C, _S = _tail_coefficients()


TWO_OVER_PI_F32 = float(np.float32(TWO_OVER_PI))
FAST_LIMIT = 2.0**18


def _lead24(x: float) -> float:
    """The leading 24 significant bits of x, truncated toward zero."""
    if x == 0.0:
        return 0.0
    m, e = math.frexp(x)
    return math.ldexp(math.trunc(m * 2.0**24) / 2.0**24, e)


def _quadrant_count(x: float) -> int:
    if abs(x) < FAST_LIMIT:
        # one FP32 FMA with the 1.5 2^23 shifter: the exact product (24 x 24 bits)
        # rounded to the nearest integer, ties to even
        return round(Fraction(_lead24(x)) * Fraction(TWO_OVER_PI_F32))
    kd = _fma64(x, TWO_OVER_PI, SHIFTER)
    return int(kd - SHIFTER)


def _cos_parts(x: float, p2: float = P2):
    k = _quadrant_count(x)
    q = k & 3
    kd = float(k)
    r = _fma64(-kd, P1, x)
    r = _fma64(-kd, p2, r)
    r2 = r * r
    rd = _split(r)
    r2d = _dmul(rd, rd)
    r4d = _dmul(r2d, r2d)
    pc, ps = _C[7], _S[7]
    for k in range(6, -1, -1):
        pc = _muladd(pc, r2d, _C[k])
        ps = _muladd(ps, r2d, _S[k])
    odd = q & 1
    t = _dmul(ps if odd else pc, r4d)
    t = _dmul(t, rd if odd else (1.0, 0.0))
    neg = q in (1, 2)
    base = r if odd else 1.0
    P = -base if neg else base
    lead = _fma64(P, r2 * (-1.0 / 6.0 if odd else -0.5), P)
    return lead, ((-t[0], -t[1]) if neg else t)


def _worst_error(xs, p2=P2):
    mpmath.mp.dps = 40
    worst = 0.0
    for x in xs:
        lead, tail = _cos_parts(float(x), p2)
        v = mpmath.mpf(lead) + mpmath.mpf(tail[0]) + mpmath.mpf(tail[1])
        worst = max(worst, abs(float(v - mpmath.cos(mpmath.mpf(float(x))))))
    return worst


def _arguments():
    rng = np.random.default_rng(1)
    xs = list(rng.uniform(-10.0, 10.0, 200)) + list(rng.uniform(-1e6, 1e6, 100))
    xs += list(10.0 ** rng.uniform(-3.0, 14.7, 200))
    xs += [0.0, math.pi / 4, math.pi / 2, -math.pi, 2.0**49 - 1.0, 1e-300]
    # near half-integers of 2x/pi below 2^18, where the FP32 quadrant count may be one off
    xs += [(kk + 0.5) * math.pi / 2 * (1.0 + d) for kk in (1000, 77777, 150000) for d in (-1e-9, 0.0, 1e-9)]
    xs += [2.0**18 * 0.999, 2.0**18 * 1.001]
    return xs


def test_fp32_quadrant_count_is_within_half_plus_two_percent():
    rng = np.random.default_rng(2)
    for x in list(rng.uniform(-FAST_LIMIT, FAST_LIMIT, 2000)) + [0.75 * FAST_LIMIT, -0.999 * FAST_LIMIT]:
        k = _quadrant_count(float(x))
        err = abs(float(x) * 2.0 / math.pi - k)
        assert err <= 0.5 + 0.02, (x, k, err)


def test_cosine_within_a_few_units_of_2_pow_minus_53():
    assert _worst_error(_arguments()) <= 4.0 * 2.0**-53


def test_one_part_reduction_is_detected():
    xs = [1e6 + 0.5, 3.0e9, 1.0e13]
    assert _worst_error(xs, p2=0.0) > 4.0 * 2.0**-53
