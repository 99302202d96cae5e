// dse_lnrcp.cuh -- ln z and 1/z of the quadrature kernels (device code).
#pragma once

#include "dse_df.cuh"
#include "dse_lntab.cuh"

namespace dse {
namespace {

// ---- ln z and 1/z (table-driven, Tang 1990) ----
// z = 2^e m with m in [1, 2); for the leading 7 fraction bits j of m, c_j =
// 1 + (j + 1/2)/128, inv_j = 1/c_j rounded to FP64 and L_j = -ln(inv_j) as a
// double-double (dse_lntab.cuh, written by gen_lntab.py with 60-digit arithmetic).
// With r = m inv_j - 1 (one FMA, |r| < 2^-7.9):
//   ln z = (e ln2_hi + L_j,hi) + r + [c + e ln2_lo + L_j,lo],
//          c = ln(1 + r) - r = -r^2 (1/2 - r/3 + r^2/4 - r^3/5 + r^4/6) (|c| < 2^-16.8);
//   1/z = 2^-e inv_j ((1 - r) + [d]),  d = 1/(1 + r) - (1 - r) = r^2 (1 - r + r^2 - r^3 + r^4);
// where the bracketed small terms are formed in double-float on the FP32 pipe (they
// need about 40 significant bits) and only the leading sums and the FMAs of r, of
// e ln2_hi and of inv_j (1 - r) + inv_j d take the FP64 pipe (8 FP64 operations; e as
// a double comes from integer operations).  ln2 = ln2_hi
// + ln2_lo with ln2_hi holding 42 significant bits, so e ln2_hi is exact.  Accuracy
// (tests/test_ln_rcp.py, an emulation of these operations against 40-digit values over
// z in [1e-14, 1e8]): ln z within 2 units of 2^-53 max(1, |ln z|), 1/z within 2 units in
// the last place.  Zero, subnormal, negative, very large, infinite and NaN arguments
// take the library routines.
constexpr int kLnTab = 128;  // g_lntab: inv_j, L_j hi, L_j lo (kLnTab each), ln2_hi, ln2_lo
constexpr float kLn2LoF = 0x1.ef357ap-45f;   // ln2_lo of g_lntab rounded to FP32
constexpr float kThirdHi = 0x1.555556p-2f;   // 1/3 = kThirdHi + kThirdLo to 2^-50
constexpr float kThirdLo = -0x1.555556p-27f;

struct LnRcp { double ln, rcp; };

__device__ __forceinline__ LnRcp ln_rcp(double z) {
    LnRcp o;
    const int hz = __double2hiint(z);
    if (hz < 0x00300000 || hz >= 0x7fc00000) {  // outside [2^-1020, 2^1021), or negative
        o.ln = log(z);
        o.rcp = 1.0 / z;
        return o;
    }
    const int e = ((hz >> 20) & 0x7ff) - 1023;
    const int j = (hz >> 13) & (kLnTab - 1);
    const double m = __hiloint2double((hz & 0x000fffff) | 0x3ff00000, __double2loint(z));
    const double inv = __ldg(&g_lntab[j]);
    const double Lh = __ldg(&g_lntab[kLnTab + j]), Ll = __ldg(&g_lntab[2 * kLnTab + j]);
    const double ln2h = __ldg(&g_lntab[3 * kLnTab]);
    const double r = fma(m, inv, -1.0);
    const float2 rd = df_split(r, 0);
    const float rf = rd.x;
    // r^2 = p2 + e2: the exact product of the leading parts and the cross term
    const float p2 = rf * rf;
    const float e2 = fmaf(2.0f * rf, rd.y, fmaf(rf, rf, -p2));
    // c = -r^2 P, P = (1/2 - r/3) + (r^2/4 - r^3/5 + r^4/6), the first part in double-float
    const float2 r3 = df_mul(rd, make_float2(kThirdHi, kThirdLo));
    const float ph = 0.5f - r3.x;
    const float pl = (((0.5f - ph) - r3.x) - r3.y) + p2 * fmaf(fmaf(1.0f / 6.0f, rf, -0.2f), rf, 0.25f);
    const float2 cm = df_mul(make_float2(p2, e2), make_float2(ph, pl));
    // S = c + e ln2_lo + L_j,lo (the last two below 2^-32: FP32 suffices)
    const float ef = __int_as_float(0x4b400000 + e) - 12582912.0f;  // e as FP32 (|e| < 2^22)
    const float sl = fmaf(ef, kLn2LoF, (float)Ll) - cm.y;
    // d = r^2 Q, Q = (1 - r) + (r^2 - r^3 + r^4), the first part in double-float
    const float qh = 1.0f - rf;
    const float ql = (((1.0f - qh) - rf) - rd.y) + p2 * (1.0f - rf + p2);
    const float2 dm = df_mul(make_float2(p2, e2), make_float2(qh, ql));
    // e as a double without a conversion instruction: 1.5 2^52 + (e + 2^31) - (1.5 2^52 + 2^31)
    const double ed = int_as_double(e);  // (integer operations, no FP64 instruction)
    const double hi = fma(ed, ln2h, Lh);
    o.ln = hi + ((r - df_widen(cm.x, 1023)) + df_widen(sl, 1023));
    // inv (1 - r + d) = inv (1 - r) + inv d: two FMAs (d exact in FP64 as hi + lo)
    const double t = fma(inv, df_widen(dm.x, 1023) + df_widen(dm.y, 1023), fma(-inv, r, inv));
    // t in (1/2, 1.004]: scaled by 2^-e in its exponent field
    o.rcp = __hiloint2double(__double2hiint(t) - (e << 20), __double2loint(t));
    return o;
}

}  // namespace
}  // namespace dse
