"""FP32 double-float arithmetic of the device kernels, emulated on the CPU for the
error-bound tests: each FP32 operation rounds once (numpy float32), FMA is exact
rational arithmetic rounded once, FP64 FMA likewise.  A value is hi + lo, two FP32
numbers (Dekker's exact product by FMA, Knuth's exact sum)."""
import math
from fractions import Fraction as Fr

import numpy as np

f32 = np.float32


def _round32(q: Fr) -> float:
    """q rounded to the nearest FP32 value (ties to even); normal range only."""
    if q == 0:
        return 0.0
    sg = -1 if q < 0 else 1
    q = abs(q)
    e = math.frexp(float(q))[1] - 1
    while Fr(2) ** e > q:
        e -= 1
    while Fr(2) ** (e + 1) <= q:
        e += 1
    sc = Fr(2) ** (23 - e)
    m = q * sc
    n = m.numerator // m.denominator
    r = m - n
    if r > Fr(1, 2) or (r == Fr(1, 2) and n % 2 == 1):
        n += 1
    return float(sg * Fr(n) / sc)


def _fmaf(a, b, c):
    return _round32(Fr(a) * Fr(b) + Fr(c))


def _add(a, b):
    return float(f32(a) + f32(b))


def _sub(a, b):
    return float(f32(a) - f32(b))


def _mul(a, b):
    return float(f32(a) * f32(b))


def _fma64(a, b, c):
    return float(Fr(a) * Fr(b) + Fr(c))  # one rounding to FP64


def _split(x: float):
    """x as hi + lo: hi the leading 24 bits (truncated), lo the rest rounded to FP32."""
    b = np.array([x]).view(np.uint64)[0]
    hi = float(np.array([b & ~np.uint64((1 << 29) - 1)], dtype=np.uint64).view(np.float64)[0])
    return hi, float(f32(x - hi))


def _mulsub(a, b, d):
    """a b - d in double-float: exact product of the leading parts, the two cross
    terms, the exact difference of the leading parts, renormalised."""
    p = _mul(a[0], b[0])
    e = _fmaf(a[0], b[0], -p)
    e = _fmaf(a[0], b[1], e)
    e = _fmaf(a[1], b[0], e)
    sm = _sub(p, d[0])
    bb = _sub(sm, p)
    err = _add(_sub(p, _sub(sm, bb)), _sub(-d[0], bb))
    lo = _sub(_add(e, err), d[1])
    hi = _add(sm, lo)
    return hi, _sub(lo, _sub(hi, sm))



def _muladd(a, b, d):
    """a b + d in double-float, renormalised."""
    p = _mul(a[0], b[0])
    e = _fmaf(a[0], b[0], -p)
    e = _fmaf(a[0], b[1], e)
    e = _fmaf(a[1], b[0], e)
    sm = _add(p, d[0])
    bb = _sub(sm, p)
    err = _add(_sub(p, _sub(sm, bb)), _sub(d[0], bb))
    lo = _add(_add(e, err), d[1])
    hi = _add(sm, lo)
    return hi, _sub(lo, _sub(hi, sm))


def _dmul(a, b):
    """a b in double-float, renormalised."""
    p = _mul(a[0], b[0])
    e = _fmaf(a[0], b[0], -p)
    e = _fmaf(a[0], b[1], e)
    e = _fmaf(a[1], b[0], e)
    hi = _add(p, e)
    return hi, _sub(e, _sub(hi, p))
