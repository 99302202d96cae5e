"""Error bound of ln z and 1/z in the quadrature kernel (ln_rcp in
paper_1206_1779_gb300/csrc/dse_lnrcp.cuh), checked on the CPU by an emulation of its
operations against 40-digit values.  s(z) = (ln z - L0)/L1 is the Chebyshev argument
of the dressing functions (Sec. 3), so ln z must be good to the FP64 level; 1/z
enters every integrand.

The kernel reduces z = 2^e m with the table of dse_lntab.cuh (r = m inv_j - 1 by one
FP64 FMA), forms the small terms c = ln(1 + r) - r and d = 1/(1 + r) - (1 - r) in
double-float (FP32 pairs) and adds them to the FP64 leading parts.  Each FP32
operation below rounds once (numpy float32), FMA is exact rational arithmetic
rounded once, FP64 operations are Python floats.  Pinned: ln z within 2 units of
2^-53 max(1, |ln z|) and 1/z within 2 units in the last place.  A dropped term of
either series, a wrong sign, or the small terms computed in plain FP32 break it.
"""
import math
import os
import re

import numpy as np
import pytest

from df_emulation import _dmul, _fmaf, _fma64, _split, f32

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_1206_1779_gb300", "csrc", "dse_lnrcp.cuh")
TAB = os.path.join(ROOT, "paper_1206_1779_gb300", "csrc", "dse_lntab.cuh")


def _table():
    body = open(TAB).read().split("{", 1)[1].split("}", 1)[0]
    return [float.fromhex(t) for t in re.findall(r"-?0x[0-9a-fp.+-]+", body)]


def _fconst(name):
    m = re.search(r"constexpr float %s = (-?0x[0-9a-fp.+-]+)f;" % name, open(SRC).read())
    assert m, name
    return float(f32(float.fromhex(m.group(1))))


def _f(x):
    return float(f32(x))


def ln_rcp(z, t, third, ln2lo_f):
    """The kernel's ln_rcp for z in [2^-1020, 2^1021), operation by operation."""
    m, e = math.frexp(z)  # z = m 2^e, m in [1/2, 1)
    m, e = 2.0 * m, e - 1
    j = int((m - 1.0) * 128)
    inv, Lh, Ll, ln2h = t[j], t[128 + j], t[256 + j], t[384]
    r = _fma64(m, inv, -1.0)
    rd = _split(r)
    rf = rd[0]
    p2 = _f(rf * rf)
    e2 = _fmaf(_f(2.0 * rf), rd[1], _fmaf(rf, rf, -p2))
    r3 = _dmul(rd, third)
    ph = _f(0.5 - r3[0])
    tail = _f(p2 * _fmaf(_fmaf(_f(1.0 / 6.0), rf, _f(-0.2)), rf, 0.25))
    pl = _f(_f(_f(_f(0.5 - ph) - r3[0]) - r3[1]) + tail)
    cm = _dmul((p2, e2), (ph, pl))
    sl = _f(_fmaf(float(e), ln2lo_f, _f(Ll)) - cm[1])
    qh = _f(1.0 - rf)
    ql = _f(_f(_f(_f(1.0 - qh) - rf) - rd[1]) + _f(p2 * _f(_f(1.0 - rf) + p2)))
    dm = _dmul((p2, e2), (qh, ql))
    hi = _fma64(float(e), ln2h, Lh)
    ln = hi + ((r - cm[0]) + sl)
    t1 = _fma64(-inv, r, inv)
    rcp = math.ldexp(_fma64(inv, dm[0] + dm[1], t1), -e)
    return ln, rcp


def test_ln_rcp_bounds():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    t = _table()
    third = (_fconst("kThirdHi"), _fconst("kThirdLo"))
    ln2lo_f = _fconst("kLn2LoF")
    assert ln2lo_f == _f(t[385])
    assert abs(mpmath.mpf(third[0]) + mpmath.mpf(third[1]) - mpmath.mpf(1) / 3) < mpmath.mpf(2) ** -50
    rng = np.random.default_rng(7)
    zs = list(np.exp(rng.uniform(math.log(1e-14), math.log(1e8), 3000)))
    # interval edges of the table and of the binades, and exact powers of two
    for j in range(128):
        for k in (-40, -1, 0, 1, 20):
            zs.append(math.ldexp(1.0 + j / 128.0, k))
            zs.append(math.ldexp(math.nextafter(1.0 + (j + 1) / 128.0, 0.0), k))
    zs += [math.ldexp(1.0, k) for k in range(-47, 27)]
    worst_ln = worst_rcp = 0.0
    for z in zs:
        if not (1.0 <= z * 2.0 ** 1020 and z < 2.0 ** 1021):
            continue
        ln, rcp = ln_rcp(z, t, third, ln2lo_f)
        L = mpmath.log(mpmath.mpf(z))
        err_ln = float(abs(mpmath.mpf(ln) - L)) / (2.0 ** -53 * max(1.0, abs(float(L))))
        R = 1 / mpmath.mpf(z)
        err_rcp = float(abs(mpmath.mpf(rcp) - R)) / math.ulp(float(R))
        worst_ln = max(worst_ln, err_ln)
        worst_rcp = max(worst_rcp, err_rcp)
    print("ln z: worst %.2f units of 2^-53 max(1, |ln z|); 1/z: worst %.2f ulp" % (worst_ln, worst_rcp))
    assert worst_ln <= 2.0
    assert worst_rcp <= 2.0
