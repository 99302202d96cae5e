// dse_df.cuh -- double-float arithmetic on the FP32 pipe: a value is the
// unevaluated sum hi + lo of two FP32 numbers (48 significant bits).  Products use
// the exact FMA product of the leading parts plus the cross terms (Dekker 1971),
// sums the exact two-sum (Knuth).  This GPU issues FP32 at 64 times its FP64
// rate, so FP64 kernels move sums whose terms need more than FP32 but less than
// FP64 precision here.
#pragma once

#include <cuda_runtime.h>

namespace dse {

// x 2^-sh as hi + lo: hi keeps the leading 24 significant bits of x (by
// truncation, so x - hi is exact), lo the next 24 (rounded).  Values below the
// FP32 normal range after scaling are flushed to zero; Inf/NaN give NaN.
__device__ __forceinline__ float2 df_split(double x, int sh) {
    const unsigned hb = (unsigned)__double2hiint(x), lb = (unsigned)__double2loint(x);
    const int e = (int)((hb >> 20) & 0x7ffu);
    if (e == 0x7ff) return make_float2(__int_as_float(0x7fc00000), 0.0f);
    const int ef = e - sh - 896;  // biased FP32 exponent of x 2^-sh
    if (e == 0 || ef < 1) return make_float2(0.0f, 0.0f);  // zero, subnormal or flushed
    const unsigned sign = hb & 0x80000000u;
    const float hi = __int_as_float((int)(sign | ((unsigned)ef << 23) | ((hb & 0xfffffu) << 3) | (lb >> 29)));
    // the 29 bits below hi: r 2^(ef - 127 - 52)
    const float lo = __uint2float_rn(lb & 0x1fffffffu) * 0x1p-52f * __int_as_float(ef << 23);
    return make_float2(hi, __int_as_float(__float_as_int(lo) | (int)sign));
}

// c += a b in double-float: exact product of the leading parts (FMA), the cross
// terms in FP32, the exact sum of c.x and the product's leading part; the lower
// parts are collected in c.y (renormalised by df_renorm).
__device__ __forceinline__ void df_fma(float2& c, const float2 a, const float2 b) {
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    const float sm = c.x + p;
    const float bb = sm - c.x;
    const float err = (c.x - (sm - bb)) + (p - bb);
    c.y += err + e;
    c.x = sm;
}

// 2 v exactly for finite |v| < 2^1023, by integer operations on its bits (the
// exponent field plus one, or the significand shifted for zero and subnormals), so
// that no FP64 instruction is spent on it.
__device__ __forceinline__ double twice(double v) {
    const int hi = __double2hiint(v);
    const unsigned lo = (unsigned)__double2loint(v);
    if (hi & 0x7ff00000) return __hiloint2double(hi + 0x00100000, (int)lo);
    const unsigned mh = ((unsigned)hi << 1) | (lo >> 31);  // (the sign bit shifts out)
    return __hiloint2double((int)((mh & 0x7fffffffu) | ((unsigned)hi & 0x80000000u)), (int)(lo << 1));
}

// An integer k (|k| < 2^31) as a double, by integer operations: the exponent from
// the position of the leading one, the bits below it as the significand.
__device__ __forceinline__ double int_as_double(int k) {
    if (k == 0) return 0.0;
    const unsigned sign = k < 0 ? 0x80000000u : 0u;
    const unsigned a = k < 0 ? 0u - (unsigned)k : (unsigned)k;
    const int lz = __clz((int)a);
    const unsigned m = (a << lz) << 1;  // the bits below the leading one, left-aligned
    return __hiloint2double((int)(sign | ((unsigned)(1054 - lz) << 20) | (m >> 12)), (int)(m << 20));
}

// f 2^(E - 1023) as a double, from the bits of f: the tile scale of phase B
// folded into the exponent (zero and FP32 subnormals give 0, Inf/NaN or an
// overflow give Inf/NaN).
__device__ __forceinline__ double df_widen(float f, int E) {
    const unsigned b = (unsigned)__float_as_int(f);
    const int e8 = (int)((b >> 23) & 0xffu);
    if (e8 == 0) return 0.0;
    int e11 = e8 + E - 127;
    if (e8 == 0xff || E == 0x7ff) e11 = 0x7ff;
    if (e11 <= 0) return 0.0;
    if (e11 > 0x7ff) e11 = 0x7ff;
    const unsigned m = b & 0x7fffffu;
    return __hiloint2double((int)((b & 0x80000000u) | ((unsigned)e11 << 20) | (m >> 3)), (int)(m << 29));
}

// a b + d in double-float (renormalised)
__device__ __forceinline__ float2 df_muladd(const float2 a, const float2 b, const float2 d) {
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    const float sm = p + d.x;
    const float bb = sm - p;
    const float err = (p - (sm - bb)) + (d.x - bb);
    const float lo = (e + err) + d.y;
    const float hi = sm + lo;
    return make_float2(hi, lo - (hi - sm));
}

// a b - d in double-float (renormalised)
__device__ __forceinline__ float2 df_mulsub(const float2 a, const float2 b, const float2 d) {
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    const float sm = p - d.x;
    const float bb = sm - p;
    const float err = (p - (sm - bb)) + (-d.x - bb);
    const float lo = (e + err) - d.y;
    const float hi = sm + lo;
    return make_float2(hi, lo - (hi - sm));
}

// a b - d in double-float, not renormalised: (sum of the leading parts, collected
// low parts), |lo| within a few units of the leading part's last place; for a value
// that only enters products as an operand
__device__ __forceinline__ float2 df_mulsub_nr(const float2 a, const float2 b, const float2 d) {
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    const float sm = p - d.x;
    const float bb = sm - p;
    const float err = (p - (sm - bb)) + (-d.x - bb);
    return make_float2(sm, (e + err) - d.y);
}

// a + b in double-float (renormalised; exact sum of the leading parts)
__device__ __forceinline__ float2 df_add(const float2 a, const float2 b) {
    const float s = a.x + b.x;
    const float bb = s - a.x;
    float e = (a.x - (s - bb)) + (b.x - bb);
    e += a.y + b.y;
    const float hi = s + e;
    return make_float2(hi, e - (hi - s));
}

__device__ __forceinline__ void df_renorm(float2& c) {
    const float sm = c.x + c.y;
    c.y = c.y - (sm - c.x);
    c.x = sm;
}

// a b in double-float (renormalised)
__device__ __forceinline__ float2 df_mul(const float2 a, const float2 b) {
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    const float hi = p + e;
    return make_float2(hi, e - (hi - p));
}

// ---- two double-float values at once, on the paired FP32 instructions of this GPU
// (f32x2: one instruction serves both lanes of a float2, each lane rounded exactly
// as the scalar instruction).  A pair of double-float values is (h, l): h holds the
// two leading parts, l the two trailing parts.  Each routine below gives, lane by
// lane, the bits of the scalar routine of the same name, with half the issued
// instructions.  Subtraction is a - b = fma(b, -1, a) (one rounding, the same
// result as the subtraction, signed zeros included).

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 neg2(float2 a) { return __fmul2_rn(a, make_float2(-1.0f, -1.0f)); }
__device__ __forceinline__ float2 bcast2(float v) { return make_float2(v, v); }

// (ch, cl) += (ah, al) (bh, bl) lane by lane (df_fma), given nbh = -bh: the
// product's leading part enters as -p = ah nbh, so that its rounding error is
// fma(ah, bh, -p) without a negation per product
__device__ __forceinline__ void df_fma2(float2& ch, float2& cl, const float2 ah, const float2 al, const float2 bh,
                                        const float2 bl, const float2 nbh) {
    const float2 np = mul2(ah, nbh);
    float2 e = fma2(ah, bh, np);
    e = fma2(ah, bl, e);
    e = fma2(al, bh, e);
    const float2 sm = sub2(ch, np);   // c + p
    const float2 bb = sub2(sm, ch);
    const float2 err = sub2(sub2(ch, sub2(sm, bb)), add2(np, bb));  // (c - (sm - bb)) + (p - bb)
    cl = add2(cl, add2(err, e));
    ch = sm;
}

// (ah, al) (bh, bl) - (dh, dl) lane by lane (df_mulsub), given nah = -ah and
// nal = -al: the rounding error of the leading product is collected negated,
// ne = -e, which fma(-a, b, p) gives exactly
__device__ __forceinline__ void df_mulsub2(const float2 ah, const float2 nah, const float2 nal, const float2 bh,
                                           const float2 bl, const float2 dh, const float2 dl, float2& rh,
                                           float2& rl) {
    const float2 p = mul2(ah, bh);
    float2 ne = fma2(nah, bh, p);
    ne = fma2(nah, bl, ne);
    ne = fma2(nal, bh, ne);
    const float2 sm = sub2(p, dh);
    const float2 bb = sub2(sm, p);
    const float2 err = sub2(sub2(p, sub2(sm, bb)), add2(dh, bb));  // (p - (sm - bb)) + (-d - bb)
    const float2 lo = sub2(sub2(err, ne), dl);                     // (e + err) - d.lo
    const float2 hi = add2(sm, lo);
    rh = hi;
    rl = sub2(lo, sub2(hi, sm));
}

// (ah, al) (bh, bl) + (dh, dl) lane by lane (df_muladd), given nbh = -bh
__device__ __forceinline__ void df_muladd2(const float2 ah, const float2 al, const float2 bh, const float2 bl,
                                           const float2 nbh, const float2 dh, const float2 dl, float2& rh,
                                           float2& rl) {
    const float2 np = mul2(ah, nbh);  // -p
    float2 e = fma2(ah, bh, np);
    e = fma2(ah, bl, e);
    e = fma2(al, bh, e);
    const float2 sm = sub2(dh, np);  // p + d
    const float2 bb = add2(sm, np);  // sm - p
    const float2 err = sub2(sub2(dh, bb), add2(np, sub2(sm, bb)));  // (p - (sm - bb)) + (d - bb)
    const float2 lo = add2(add2(e, err), dl);
    const float2 hi = add2(sm, lo);
    rh = hi;
    rl = sub2(lo, sub2(hi, sm));
}

// df_renorm on both lanes
__device__ __forceinline__ void df_renorm2(float2& ch, float2& cl) {
    const float2 sm = add2(ch, cl);
    cl = sub2(cl, sub2(sm, ch));
    ch = sm;
}

}  // namespace dse
