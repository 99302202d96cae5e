"""Host-side pin for the logarithm table of the quadrature kernel
(paper_1206_1779_gb300/csrc/dse_lntab.cuh): inv_j = 1/c_j rounded to FP64 with
c_j = 1 + (j + 1/2)/128, L_j = -ln(inv_j) as a double-double, and the split
ln 2 = ln2_hi + ln2_lo with 42 significant bits in ln2_hi, against 50-digit
arithmetic."""
import os
import re
import struct

import pytest

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_1206_1779_gb300", "csrc", "dse_lntab.cuh")


def table():
    body = open(HDR).read().split("{", 1)[1].split("}", 1)[0]
    return [float.fromhex(t) for t in re.findall(r"-?0x[0-9a-fp.+-]+", body)]


def test_lntab_values():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    t = table()
    assert len(t) == 3 * 128 + 2
    for j in range(128):
        cj = 1 + (mpmath.mpf(j) + mpmath.mpf(1) / 2) / 128
        inv = t[j]
        assert inv == float(1 / cj)
        L = -mpmath.log(mpmath.mpf(inv))
        assert t[128 + j] == float(L)
        assert abs(mpmath.mpf(t[128 + j]) + mpmath.mpf(t[256 + j]) - L) < mpmath.mpf(2) ** -105
        # the reduced argument stays below 2^-7.9 for every m of the interval
        for m in (1 + mpmath.mpf(j) / 128, 1 + mpmath.mpf(j + 1) / 128):
            assert abs(m * mpmath.mpf(inv) - 1) < mpmath.mpf(2) ** -7.9
    ln2_hi, ln2_lo = t[384], t[385]
    bits = struct.unpack("<Q", struct.pack("<d", ln2_hi))[0]
    assert bits & ((1 << 11) - 1) == 0  # e ln2_hi exact for |e| < 2^11
    assert abs(mpmath.mpf(ln2_hi) + mpmath.mpf(ln2_lo) - mpmath.log(2)) < mpmath.mpf(2) ** -95
