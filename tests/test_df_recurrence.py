"""Error bound of the double-float Chebyshev values of the hot kernel (Sec. 3 basis
T_j(s)), checked on the CPU by an emulation of the arithmetic against 50-digit values.

The kernel represents a value as hi + lo, two FP32 numbers.  It forms the anchors
T_4i, T_4i+1 by the stride-4 recurrence X_(i+1) = 2 T_4 X_i - X_(i-1), starting from
T_4 and T_5 evaluated in FP64, and the values T_4i+2, T_4i+3 by two steps of
T_(j+1) = 2 s T_j - T_(j-1).  The emulation below performs each FP32 operation of
that scheme in numpy float32.  FMA is emulated with exact rational arithmetic and one
rounding.  The test pins two bounds that the parity bar for the Newton matrix relies
on:
  - an anchor at i steps errs by at most 2 i^2 2^-48 (+ 2^-47 for the start);
  - every T_j (j < 64) errs by at most 2 (j^2 2^-49 + 2^-48), the rounding of s to
    48 bits (2^-49 relative) moved by a slope |T_j'| <= j^2.
A dropped cross term, a wrong sign in the exact sums, or the FP64 anchors replaced by
plain FP32 ones would break one of them.
"""
import numpy as np
import pytest

from df_emulation import _add, _fmaf, _fma64, _mul, _mulsub, _split, _sub

mpmath = pytest.importorskip("mpmath")


def _values(s: float, N: int):
    nq = (N + 3) // 4
    fs = _split(s)
    T2 = _fma64(2 * s, s, -1.0)
    T3 = _fma64(2 * s, T2, -s)
    T4 = _fma64(2 * T2, T2, -1.0)
    c4 = _split(2 * T4)
    a0, a1 = (1.0, 0.0), _split(T4)
    b0, b1 = fs, _split(_fma64(2 * s, T4, -T3))
    T = {0: (1.0, 0.0), 1: fs}
    for i in range(1, nq):
        T[4 * i], T[4 * i + 1] = a1, b1
        a0, a1 = a1, _mulsub(c4, a1, a0)
        b0, b1 = b1, _mulsub(c4, b1, b0)
    s2 = (2 * fs[0], 2 * fs[1])
    for i in range(nq):
        a, b = T[4 * i], T[4 * i + 1]
        t2 = _mulsub(s2, b, a)
        T[4 * i + 2] = t2
        T[4 * i + 3] = _mulsub(s2, t2, b)
    return {j: v for j, v in T.items() if j < N}


def test_double_float_chebyshev_values_within_bounds():
    mpmath.mp.dps = 50
    N = 64
    rng = np.random.default_rng(0)
    ss = [float(x) for x in rng.uniform(-1.0, 1.0, 40)]
    ss += [1.0, -1.0, 1.0 - 2.0**-30, -1.0 + 2.0**-30, 1.0 - 1e-6, -1.0 + 1e-6, 0.0, 0.5, -0.75]
    for s in ss:
        th = mpmath.acos(mpmath.mpf(s))
        for j, (hi, lo) in _values(s, N).items():
            err = abs(float(mpmath.mpf(hi) + mpmath.mpf(lo) - mpmath.cos(j * th)))
            assert err <= 2.0 * (j * j * 2.0**-49 + 2.0**-48), (s, j, err)
            if j >= 4 and j % 4 in (0, 1):
                i = j // 4
                assert err <= 2.0 * i * i * 2.0**-48 + 2.0**-47, (s, j, err)


def test_emulation_detects_a_dropped_cross_term():
    # the same check with one cross term of the product left out fails: the bound
    # is tight enough to see it
    global _mulsub
    good = _mulsub

    def bad(a, b, d):
        p = _mul(a[0], b[0])
        e = _fmaf(a[0], b[0], -p)
        e = _fmaf(a[0], b[1], e)  # a.y b.x dropped
        sm = _sub(p, d[0])
        bb = _sub(sm, p)
        err = _add(_sub(p, _sub(sm, bb)), _sub(-d[0], bb))
        lo = _sub(_add(e, err), d[1])
        hi = _add(sm, lo)
        return hi, _sub(lo, _sub(hi, sm))

    _mulsub = bad
    try:
        mpmath.mp.dps = 50
        worst = 0.0
        for s in (0.3, -0.8, 0.97, 1.0 - 1e-6):
            th = mpmath.acos(mpmath.mpf(s))
            for j, (hi, lo) in _values(s, 64).items():
                err = abs(float(mpmath.mpf(hi) + mpmath.mpf(lo) - mpmath.cos(j * th)))
                worst = max(worst, err / (2.0 * (j * j * 2.0**-49 + 2.0**-48)))
        assert worst > 1.0
    finally:
        _mulsub = good
