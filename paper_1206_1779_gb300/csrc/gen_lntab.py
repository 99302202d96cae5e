"""Writes dse_lntab.cuh: the table of the quadrature kernel's logarithm
(dse_triple.cu, ln_rcp): for j < 128, c_j = 1 + (j + 1/2)/128, inv_j = 1/c_j
rounded to FP64, and L_j = -ln(inv_j) as a double-double (hi, lo); then
ln 2 = ln2_hi + ln2_lo with ln2_hi holding the leading 42 significant bits.
Computed with 60-digit arithmetic (mpmath).  Run: python gen_lntab.py"""
import os
import struct

import mpmath

mpmath.mp.dps = 60
N = 128


def hexd(x: float) -> str:
    return float.hex(x)


inv, hi, lo = [], [], []
for j in range(N):
    cj = 1 + (mpmath.mpf(j) + mpmath.mpf(1) / 2) / N
    iv = float(1 / cj)
    L = -mpmath.log(mpmath.mpf(iv))
    h = float(L)
    inv.append(iv)
    hi.append(h)
    lo.append(float(L - mpmath.mpf(h)))
ln2 = mpmath.log(2)
b = struct.unpack("<Q", struct.pack("<d", float(ln2)))[0] & ~((1 << 11) - 1)
ln2_hi = struct.unpack("<d", struct.pack("<Q", b))[0]
ln2_lo = float(ln2 - mpmath.mpf(ln2_hi))
vals = inv + hi + lo + [ln2_hi, ln2_lo]
lines = ["// dse_lntab.cuh -- written by gen_lntab.py (do not edit): inv_j, L_j hi, L_j lo",
         "// for j < 128, then ln2_hi, ln2_lo; see ln_rcp in dse_triple.cu.",
         "#pragma once", "", "namespace dse {", "namespace {",
         "__device__ const double g_lntab[%d] = {" % len(vals)]
for k in range(0, len(vals), 3):
    lines.append("    " + ", ".join(hexd(v) for v in vals[k:k + 3]) + ",")
lines += ["};", "}  // namespace", "}  // namespace dse", ""]
out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "dse_lntab.cuh")
open(out, "w").write("\n".join(lines))
print("wrote", out)
