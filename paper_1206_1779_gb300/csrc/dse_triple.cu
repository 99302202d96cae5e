// dse_triple.cu -- the fused radial x angular quadrature kernel (the hot path).
//
// For every triple (external momentum x_r, radial node y_k, angular node theta_l)
// it forms z = x + y - 2 sqrt(xy) cos(theta) (as d + 2 b sin^2(theta/2)), evaluates
// ln G(z), ln Z(z) by the Chebyshev recurrence (Sec. 3; IR/UV forms of Sec. 2
// outside [eps2, lambda2]) and the three integrands of the ghost and gluon
// equations of Sec. 2:
//   hQ = W_k w_l sin^2 Q W                 (gluon loop, vertex model W)
//   hM = W_k w_l sin^2 M G(y) G(z)         (ghost loop in the gluon equation)
//   hG = W_k w_l y G(y) sin^4 Z(z)/z^2     (ghost equation)
// with M = y sin^2/z and Q = quartic(sin^2(theta/2))/(2 z^2), the cancellation-free
// forms of the printed kernels.  Outputs per block:
//   Upart[r][k][chunk][3]  warp-shuffle sums over 32 angular nodes of (hQ, hM, hG);
//   Vpart[r][split][3][N]  sums of (hQ, hM, hG) * phi_j(z) over the block's triples
// (FULL mode only).  The phi_j(y) part of the Newton-matrix entries depends on y
// alone and is contracted from Upart afterwards.
//
// Data flow per tile of BT triples (one warp = 32 angular nodes of one radial node):
//   phase A: each thread builds its triple in FP64, stores phi_j(z) (j < N) into
//            a shared-memory row and its three weights;
//   phase B: thread (group g, coefficient j) accumulates weight * phi_j(z) over
//            its group's rows: three multiply-adds per (triple, j).
// Phase B runs in double-float arithmetic (a value is an unevaluated sum hi + lo
// of two FP32 numbers, 48 significant bits; Dekker's exact product and Knuth's
// exact sum), because this GPU issues FP32 at 64 times its FP64 rate: the
// Chebyshev values phi_j(z) come from double-float recurrences started from FP64
// values, the FP64 weights are split exactly into (hi, lo) pairs (scaled by a
// power of two per tile, so that no tile over- or underflows FP32), each group
// sums at most one tile's rows in double-float, and the tile sums are added to
// FP64 accumulators.  The residual (the angular sums of the weights) stays in
// FP64 throughout.
// The block's coefficient vector lives in shared memory (broadcast reads).
#include "dse_df.cuh"
#include "dse_internal.cuh"
#include "dse_lnrcp.cuh"

namespace dse {

namespace {

constexpr unsigned kFullMask = 0xffffffffu;
constexpr double kPi = 3.14159265358979323846264338327950288;

__host__ __device__ inline int block_threads_for(int N) { return N <= 96 ? 128 : 64; }

// Z(z), G(z) (zg) and W(z) (w) from the series-table record R at u = uf
// (double-float): Horner over the kSeriesQ coefficients of each, the terms of
// degree >= kf in FP32 on the leading parts (the record's tail is small enough
// for that: kf = R->ex[3], here the largest over the lanes that evaluate together,
// so that they take the same steps), the rest in double-float; Z and G as the two
// lanes of paired FP32 instructions.  Results as double-float mantissas Zm, Gm, Wm
// and exponent shifts (Z = Zm 2^Zs).
__device__ __forceinline__ void series_eval_df(const SeriesRec* __restrict__ R, const float2 uf, const bool zg,
                                               const bool w, float2& Zm, float2& Gm, float2& Wm, int& Zs, int& Gs,
                                               int& Ws) {
    const int kf = __reduce_max_sync(__activemask(), __ldg(&R->ex[3]));
    // (kf is the same on every lane: two loops, the FP32 tail from degree
    // kSeriesP - 1 down to kf, then the double-float steps, instead of a branch
    // per degree)
    if (zg) {
        const float4 top = __ldg(&R->e[kSeriesP]);  // (Z hi, G hi, Z lo, G lo)
        float2 th = make_float2(top.x, top.y);
        float2 tl = kf > kSeriesP ? make_float2(top.z, top.w) : make_float2(0.0f, 0.0f);
        const float2 uh = bcast2(uf.x), ul = bcast2(uf.y), nuh = bcast2(-uf.x);
        int k = kSeriesP - 1;
#pragma unroll 4
        for (; k >= kf; --k) {
            const float4 ck = __ldg(&R->e[k]);
            th = fma2(th, uh, make_float2(ck.x, ck.y));
        }
#pragma unroll 4
        for (; k >= 0; --k) {
            const float4 ck = __ldg(&R->e[k]);
            df_muladd2(th, tl, uh, ul, nuh, make_float2(ck.x, ck.y), make_float2(ck.z, ck.w), th, tl);
        }
        const int2 ex = __ldg(reinterpret_cast<const int2*>(R->ex));
        Zm = make_float2(th.x, tl.x);
        Gm = make_float2(th.y, tl.y);
        Zs = ex.x - 1023;
        Gs = ex.y - 1023;
    }
    if (w) {
        const float2 top = __ldg(&R->w[kSeriesP]);
        float2 tw = make_float2(top.x, kf > kSeriesP ? top.y : 0.0f);
        int k = kSeriesP - 1;
#pragma unroll 4
        for (; k >= kf; --k) tw.x = fmaf(tw.x, uf.x, __ldg(&R->w[k]).x);
#pragma unroll 4
        for (; k >= 0; --k) tw = df_muladd(tw, uf, __ldg(&R->w[k]));
        Wm = tw;
        Ws = __ldg(&R->ex[2]) - 1023;
    }
}

// The same, widened to FP64.
__device__ __forceinline__ void series_eval(const SeriesRec* __restrict__ R, const float2 uf, const bool zg,
                                            const bool w, double& Z, double& G, double& W) {
    float2 Zm, Gm, Wm;
    int Zs = 0, Gs = 0, Ws = 0;
    series_eval_df(R, uf, zg, w, Zm, Gm, Wm, Zs, Gs, Ws);
    if (zg) {
        Z = df_widen(Zm.x, Zs + 1023) + df_widen(Zm.y, Zs + 1023);
        G = df_widen(Gm.x, Gs + 1023) + df_widen(Gm.y, Gs + 1023);
    }
    if (w) W = df_widen(Wm.x, Ws + 1023) + df_widen(Wm.y, Ws + 1023);
}

// The anchors T_4i, T_4i+1 for i = 1 .. nq - 1 by the recurrence of stride 4,
// X_(i+1) = 2 T_4 X_i - X_(i-1) (from T_(m+4) + T_(m-4) = 2 T_4 T_m), in
// double-float from T_4 and T_5 formed in FP64 from s (their rounding to 48 bits,
// 2^-49 relative, is the start error, which grows at most like i over i steps; the
// steps' own rounding errors, 2^-48 each, at most like i^2); the two sequences
// run as the two lanes of paired FP32 instructions; dst[i - 1] = (T_4i hi,
// T_4i+1 hi, T_4i lo, T_4i+1 lo), so that phase B loads both as one pair.  sd is s
// as a double-float pair.
__device__ __forceinline__ void store_anchors(const double s, const float2 sd, const int nq,
                                              float4* __restrict__ dst) {
    // (the doublings by integer operations: four FMAs on the FP64 pipe)
    const double s2 = twice(s);
    const double T2 = fma(s2, s, -1.0);
    const double T3 = fma(s2, T2, -s);
    const double T4 = fma(twice(T2), T2, -1.0);
    const float2 t4 = df_split(T4, 0), t5 = df_split(fma(s2, T4, -T3), 0);
    const float2 c4 = make_float2(2.0f * t4.x, 2.0f * t4.y);  // 2 T4 (exact scaling)
    const float2 ch = bcast2(c4.x), nch = bcast2(-c4.x), ncl = bcast2(-c4.y);
    float2 x0h = make_float2(1.0f, sd.x), x0l = make_float2(0.0f, sd.y);  // (T_0, T_1)
    float2 x1h = make_float2(t4.x, t5.x), x1l = make_float2(t4.y, t5.y);  // (T_4, T_5)
    for (int i = 1; i < nq; ++i) {
        dst[i - 1] = make_float4(x1h.x, x1h.y, x1l.x, x1l.y);
        float2 xnh, xnl;
        df_mulsub2(ch, nch, ncl, x1h, x1l, x0h, x0l, xnh, xnl);
        x0h = x1h;
        x0l = x1l;
        x1h = xnh;
        x1l = xnl;
    }
}

// 2^d as FP32 for -126 <= d <= 127 (0 below, Inf above)
__device__ __forceinline__ float pow2f(int d) {
    return d < -126 ? 0.0f : d > 127 ? __int_as_float(0x7f800000) : __int_as_float((127 + d) << 23);
}

// ---- single-problem kernels ----
// Radial nodes whose per-node factors are formed together (by one warp), and the
// factors per node: d, 4 sqrt(xy), K = W_k y G(y), the five quartic coefficients
// of the gluon-loop kernel.
constexpr int kRadGroup = 32;
constexpr int kRadFactors = 8;

// (x, y) factors of the integrands of radial node kq, formed once per node instead
// of per triple: z = d + b2 sigma with d = (sqrt x - sqrt y)^2, b2 = 4 sqrt(xy);
// K = W_k y G(y) (hM = K w s4 G(z)/z, hG = K w s4 Z(z)/z^2); the quartic of the
// gluon-loop kernel times W_k W(y)/2 (hQ = w s2 W(z)/z^2 sum_i kQ_i sigma^i).
__device__ __forceinline__ void radial_factors(const TripleArgs& A, const Row& row, const int rt, const int kq,
                                               double* __restrict__ f) {
    const Consts& c = A.c;
    const Rad rd = A.rad[rad_offset(c, rt) + kq];
    const YTab yt = A.ytab[rad_offset(c, rt) + kq];
    const double d0 = row.sx - rd.sy;
    const double d = d0 * d0;
    const double b = 2.0 * row.sx * rd.sy;
    f[0] = d;
    f[1] = 2.0 * b;
    f[2] = rd.W * yt.yG;
    const double dd = d * d, db = d * b, bb = b * b;
    const double h = 0.5 * rd.W * yt.Wy;
    f[3] = h * (7.5 * dd);
    f[4] = h * -(48.0 * dd + 18.0 * db + 12.0 * bb);
    f[5] = h * (48.0 * dd - 48.0 * db - 38.0 * bb);
    f[6] = h * (96.0 * db + 64.0 * bb);
    f[7] = h * (16.0 * bb);
}

// The three integrands (hQ, hM, hG) of the triple (x_r, y_k, theta_l) in FP64 and
// s(z): z = d + b2 sigma_l from the node factors f, ln z and 1/z (ln_rcp), s(z)
// (clamped outside [eps2, lambda2]), Z(z), G(z), W(z) from the series table, or by
// the per-triple series and the IR/UV forms, and the kernels M and Q.
struct TripleW {
    double hQ, hM, hG, s;
    float2 sd;  // s as a double-float pair (48 bits)
};

__device__ __forceinline__ TripleW triple_weights(const TripleArgs& A, const bool gluon, const bool ghost,
                                                  const double* __restrict__ f, const int l,
                                                  const double* __restrict__ sa, const double* __restrict__ sb,
                                                  const double* __restrict__ sbnd, const float ith_scale) {
    const Consts& c = A.c;
    const int N = c.N;
    TripleW o;
    o.hQ = o.hM = o.hG = 0.0;
    o.sd = make_float2(0.0f, 0.0f);
    const Ang an = A.ang[l];
    const double z = fma(f[1], an.sig, f[0]);
    const LnRcp lr = ln_rcp(z);
    const double lz = lr.ln;
    // s(z) = ln z / L1 - L0 / L1 (one FMA; the same value as (ln z - L0) / L1 rounded
    // twice when L0 = 0, i.e. eps2 lambda2 = 1), clamped to [-1, 1] for z outside
    // [eps2, lambda2] (inside, it can leave the interval only by a rounding)
    double s = fma(lz, c.invL1, c.sL0);
    const double iz = lr.rcp;
    const double iz2 = iz * iz;
    double Zz = 0.0, Gz = 0.0, Wz = 0.0;  // Z(z), G(z), W(z) = G(z)^p Z(z)^q
    // z > 0: the comparisons with eps2, lambda2 on the bit patterns
    const long long zb = __double_as_longlong(z);
    const bool beyond = zb < __double_as_longlong(c.eps2) || zb > __double_as_longlong(c.lam2);
    const bool outside = c.extrap == 0 && beyond;
    // beyond the range s is +-1 exactly (s of the clamped z), chosen on the integer
    // comparison (no FP64 operation)
    if (beyond) s = zb > __double_as_longlong(c.lam2) ? 1.0 : -1.0;
    const float2 sd = df_split(s, 0);  // (also the anchors' s)
    o.sd = sd;
    if (A.stab && !outside) {
        // from the table: the interval by arccos in FP32 (FP32 s from the bits of s,
        // truncated: the interval only; a neighbouring interval is as good), the
        // polynomials in double-float
        const float sf = fminf(1.0f, fmaxf(-1.0f, sd.x));
        int it = (int)(acosf(sf) * ith_scale);
        it = min(max(it, 0), c.sM - 1);
        const SeriesRec* Rr = A.stab + it;
        const double2 mh = __ldg(reinterpret_cast<const double2*>(Rr));
        series_eval(Rr, df_split((s - mh.x) * mh.y, 0), ghost || gluon, gluon, Zz, Gz, Wz);
    } else {
        double lg, lzz;
        if (A.stab) {
            // outside [eps2, lambda2]: the series at s = +-1 (block sums)
            lzz = s > 0.0 ? sbnd[0] : sbnd[2];
            lg = s > 0.0 ? sbnd[1] : sbnd[3];
        } else {
            lg = 0.5 * sb[0];
            lzz = 0.5 * sa[0];
            if (N > 1) {
                lg = fma(sb[1], s, lg);
                lzz = fma(sa[1], s, lzz);
            }
            double t0 = 1.0, t1 = s;
            const double s2x = 2.0 * s;
            for (int j = 2; j < N; ++j) {
                const double t2 = fma(s2x, t1, -t0);
                t0 = t1;
                t1 = t2;
                lg = fma(sb[j], t2, lg);
                lzz = fma(sa[j], t2, lzz);
            }
        }
        if (outside) {
            if (z < c.eps2) {
                const double r = lz - c.ln_eps2;
                lg = fma(-c.kappa, r, lg);
                lzz = fma(2.0 * c.kappa, r, lzz);
            } else {
                const double L = log1p(c.omega * (lz - c.ln_lam2));
                lg = fma(c.delta, L, lg);
                lzz = fma(c.gam, L, lzz);
            }
        }
        if (ghost) Zz = exp(lzz);
        if (gluon) {
            Gz = exp(lg);
            Wz = exp(c.pG * lg + c.qZ * lzz);
        }
    }
    const double Kw = f[2] * an.ws4;
    if (ghost) o.hG = Kw * Zz * iz2;
    if (gluon) {
        const double sg = an.sig;
        const double num = fma(sg, fma(sg, fma(sg, fma(sg, f[7], f[6]), f[5]), f[4]), f[3]);
        o.hQ = an.ws2 * iz2 * Wz * num;
        o.hM = Kw * iz * Gz;
    }
    o.s = s;
    return o;
}

// Angular sums over the warp's 32 nodes (same radial node for the whole warp) of
// (hQ, hM, hG) by halving exchanges, 6 FP64 additions per lane: lanes 0-15 go on
// with (hQ, hM), lanes 16-31 with (hG, 0); then lanes with bit 3 set with the second
// of the two; then three butterfly steps.  The sums end in lanes 0 (hQ), 8 (hM) and
// 16 (hG), which write them to up[0..2] (when write is set).
__device__ __forceinline__ void angular_sums(const TripleW& w, const int lane, const bool write, double* up) {
    const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0;
    const double k0s = (h16 ? w.hG : w.hQ) + __shfl_xor_sync(kFullMask, h16 ? w.hQ : w.hG, 16);
    const double k1s = (h16 ? 0.0 : w.hM) + __shfl_xor_sync(kFullMask, h16 ? w.hM : 0.0, 16);
    double v = (h8 ? k1s : k0s) + __shfl_xor_sync(kFullMask, h8 ? k0s : k1s, 8);
    v += __shfl_xor_sync(kFullMask, v, 4);
    v += __shfl_xor_sync(kFullMask, v, 2);
    v += __shfl_xor_sync(kFullMask, v, 1);
    if (write && (lane & 7) == 0 && lane < 24) up[lane >> 3] = v;
}

__host__ __device__ inline size_t smem_res_doubles(int N, int KB) {
    // 2 N coefficients, 4 boundary sums, the factors of a group of radial nodes
    const int kg = KB < kRadGroup ? KB : kRadGroup;
    return 2u * (size_t)N + 4u + (size_t)kg * kRadFactors;
}

// Residual mode (Upart only): one block of BT threads per (row, radial split).
template <int BT>
__device__ __forceinline__ void triple_tile_residual(const TripleArgs& A, const int rt, const int ks, double* smem) {
    const Consts& c = A.c;
    const int N = c.N;
    constexpr int WARPS = BT / 32;
    double* sa = smem;
    double* sb = sa + N;
    double* sbnd = sb + N;
    double* srad = sbnd + 4;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    for (int j = tid; j < N; j += BT) {
        sa[j] = j < c.NZ ? A.coef[j] : 0.0;
        sb[j] = j < c.NG ? A.coef[c.NZ + j] : 0.0;
    }
    const Row row = A.rows[rt];
    const bool gluon = (row.flags & kRowGluon) != 0;
    const bool ghost = (row.flags & kRowGhost) != 0;
    const int k0 = ks * A.KB;
    const int k1 = min(c.nr, k0 + A.KB);
    const int nch = A.nch;
    const int nunits = k1 > k0 ? (k1 - k0) * nch : 0;
    const int kgrp = A.KB < kRadGroup ? A.KB : kRadGroup;
    const float ith_scale = (float)c.sM * (float)(1.0 / kPi);
    if (A.stab && tid < 4) sbnd[tid] = reinterpret_cast<const double*>(A.stab + kSeriesM)[tid];
    // a group of kgrp nodes spans whole tiles when kgrp = kRadGroup (kRadGroup nch is
    // a multiple of WARPS); with fewer nodes per block one group covers the block
    const int group_units = kgrp * nch;
    for (int base = 0; base < nunits; base += WARPS) {
        if (base % group_units == 0) {
            __syncthreads();  // the previous group's factors are no longer read (and the coefficients staged)
            if (warp == 0 && lane < kgrp && k0 + base / nch + lane < k1)
                radial_factors(A, row, rt, k0 + base / nch + lane, srad + lane * kRadFactors);
            __syncthreads();
        }
        const int u = base + warp;
        TripleW w;
        w.hQ = w.hM = w.hG = w.s = 0.0;
        int k = 0, ch = 0;
        if (u < nunits) {
            const int kk = u / nch;
            ch = u - kk * nch;
            k = k0 + kk;
            const int l = ch * 32 + lane;
            if (l < c.na)
                w = triple_weights(A, gluon, ghost, srad + (kk % kgrp) * kRadFactors, l, sa, sb, sbnd, ith_scale);
        }
        angular_sums(w, lane, u < nunits, A.Upart + (((size_t)rt * c.nr + k) * nch + ch) * 3);
    }
}

// ---- Newton-matrix mode ----
// One block of BT threads per (row, radial split); tiles of BT triples (one warp =
// 32 angular nodes of one radial node), each in two phases separated by barriers:
//   phase A: each thread forms its triple's FP64 weights and s(z) (triple_weights),
//            the warp's angular sums (Upart), and its shared-memory row;
//   phase B: the derivative sums weight * T_j(s) in double-float on the FP32 pipe.
// Shared-memory row of triple m (float4 units, stride rs4 = quad_count(N) + 1 made
// odd, so that the rows of eight consecutive triples fall in distinct banks):
//   [0] (2s, hQ), [1] (hM, hG) as double-float pairs, the weights times 2^-E with E
//       the block's running exponent of each weight kind;
//   [1 + i] (T_4i, T_4i+1) for quads i = 1 .. nq - 1 (quad 0 is T_0 = 1, T_1 = s).
// Phase B: thread (group g, quad i) owns the columns j = 4i .. 4i+3 and the rows of
// group g; it forms T_4i+2, T_4i+3 by two double-float steps of the recurrence and
// adds the twelve products weight * T_j to double-float accumulators that live for
// the whole block, at the block's running scale.
__host__ __device__ inline int quad_count(int N) { return (N + 3) / 4; }
__host__ __device__ inline int row_stride4(int N) { return (quad_count(N) + 1) | 1; }

__host__ __device__ inline size_t tile_full_doubles(int N, int BT) {
    const size_t t = 2u * (size_t)BT * (size_t)row_stride4(N);  // float4 = 2 doubles
    const size_t red = (size_t)(BT / quad_count(N)) * 3u * (size_t)N;  // groups' sums, float2 = 1 double
    return t > red ? t : red;
}

__host__ __device__ inline size_t smem_full_doubles(int N, int BT, int KB) {
    // tile rows, 2 N coefficients, 4 boundary sums, 8 (16 ints: per-warp exponents),
    // the factors of a group of radial nodes
    const int kg = KB < kRadGroup ? KB : kRadGroup;
    return tile_full_doubles(N, BT) + 2u * (size_t)N + 4u + 8u + (size_t)kg * kRadFactors;
}

template <int BT>
__device__ __forceinline__ void triple_tile_full(const TripleArgs& A, const int rt, const int ks, double* smem) {
    const Consts& c = A.c;
    const int N = c.N;
    const int nq = quad_count(N);
    const int rs4 = row_stride4(N);
    constexpr int WARPS = BT / 32;
    static_assert(WARPS <= 4, "per-warp exponents hold 4 warps");
    float4* sT = reinterpret_cast<float4*>(smem);
    double* sa = smem + tile_full_doubles(N, BT);
    double* sb = sa + N;
    double* sbnd = sb + N;  // ln Z(s=1), ln G(s=1), ln Z(s=-1), ln G(s=-1) (table path)
    int* sE = reinterpret_cast<int*>(sbnd + 4);  // [WARPS][4] per-warp maxima of the weights' exponents
    double* srad = sbnd + 12;                    // [min(KB, kRadGroup)][kRadFactors] radial-node factors
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;

    for (int j = tid; j < N; j += BT) {
        sa[j] = j < c.NZ ? A.coef[j] : 0.0;
        sb[j] = j < c.NG ? A.coef[c.NZ + j] : 0.0;
    }
    if (A.stab && tid < 4) sbnd[tid] = reinterpret_cast<const double*>(A.stab + kSeriesM)[tid];
    const Row row = A.rows[rt];
    const bool gluon = (row.flags & kRowGluon) != 0;
    const bool ghost = (row.flags & kRowGhost) != 0;
    const int k0 = ks * A.KB;
    const int k1 = min(c.nr, k0 + A.KB);
    const int nch = A.nch;
    const int nunits = k1 > k0 ? (k1 - k0) * nch : 0;
    const int kgrp = A.KB < kRadGroup ? A.KB : kRadGroup;
    const float ith_scale = (float)c.sM * (float)(1.0 / kPi);

    // phase-B mapping: G groups of nq threads, rows [g R, (g + 1) R)
    const int G = BT / nq;
    const int R = (BT + G - 1) / G;
    const int g = tid / nq;
    const int qi = tid - g * nq;
    const bool bact = g < G;
    const int mlo = min(BT, g * R);
    const int mhi = min(BT, mlo + R);
    // accumulators: kind kd, columns (4 qi, 4 qi + 1) in accH/accL[kd][0] and
    // (4 qi + 2, 4 qi + 3) in [kd][1], leading parts in H, trailing in L (the lanes of
    // the paired instructions)
    float2 accH[3][2], accL[3][2];
#pragma unroll
    for (int kd = 0; kd < 3; ++kd)
#pragma unroll
        for (int q = 0; q < 2; ++q) accH[kd][q] = accL[kd][q] = make_float2(0.0f, 0.0f);
    int Erun[3] = {0, 0, 0};  // running biased exponents of the accumulators' scale (0: nothing yet)

    // a group of kgrp nodes spans whole tiles when kgrp = kRadGroup (kRadGroup nch is
    // a multiple of WARPS); with fewer nodes per block one group covers the block
    const int group_units = kgrp * nch;
    // this warp's unit u = base + warp as (radial node kk, angular chunk ch), and the
    // first node of the current group, kept by increments (no integer divisions)
    int kk = warp / nch, ch = warp - (warp / nch) * nch;
    int gnode = -kgrp, next_group = 0;
    for (int base = 0; base < nunits; base += WARPS) {
        if (base == next_group) {
            next_group += group_units;
            gnode += kgrp;
            __syncthreads();  // the previous group's factors are no longer read (and the coefficients staged)
            if (warp == 0 && lane < kgrp && k0 + gnode + lane < k1)
                radial_factors(A, row, rt, k0 + gnode + lane, srad + lane * kRadFactors);
            __syncthreads();
        }
        const int u = base + warp;
        TripleW w;
        w.hQ = w.hM = w.hG = w.s = 0.0;
        w.sd = make_float2(0.0f, 0.0f);
        bool live = false;
        const int k = k0 + kk;
        if (u < nunits) {
            const int l = ch * 32 + lane;
            if (l < c.na) {
                live = true;
                w = triple_weights(A, gluon, ghost, srad + (kk - gnode) * kRadFactors, l, sa, sb, sbnd, ith_scale);
            }
        }
        angular_sums(w, lane, u < nunits, A.Upart + (((size_t)rt * c.nr + k) * nch + ch) * 3);
        // the next unit of this warp
        ch += WARPS;
        while (ch >= nch) {
            ch -= nch;
            ++kk;
        }
        float4* Trow = sT + tid * rs4;
        const float2 sd = w.sd;  // s as a double-float pair (48 bits)
        if (live) {
            store_anchors(w.s, sd, nq, Trow + 2);
        } else {
            for (int i = 1; i < nq; ++i) Trow[1 + i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
        // per-warp maxima of the weights' exponents
        {
            const unsigned eq = ((unsigned)__double2hiint(w.hQ) >> 20) & 0x7ffu;
            const unsigned em = ((unsigned)__double2hiint(w.hM) >> 20) & 0x7ffu;
            const unsigned eg = ((unsigned)__double2hiint(w.hG) >> 20) & 0x7ffu;
            const unsigned mq = __reduce_max_sync(kFullMask, eq);
            const unsigned mm = __reduce_max_sync(kFullMask, em);
            const unsigned mg = __reduce_max_sync(kFullMask, eg);
            if (lane == 0) {
                sE[warp * 4 + 0] = (int)mq;
                sE[warp * 4 + 1] = (int)mm;
                sE[warp * 4 + 2] = (int)mg;
            }
        }
        __syncthreads();
        // the block's running scale per weight kind: the largest exponent so far;
        // when it grows, the accumulators are rescaled (exact powers of two)
#pragma unroll
        for (int kd = 0; kd < 3; ++kd) {
            int Et = sE[kd];
#pragma unroll
            for (int ww = 1; ww < WARPS; ++ww) Et = max(Et, sE[ww * 4 + kd]);
            if (Et > Erun[kd]) {
                const float2 f = bcast2(pow2f(Erun[kd] - Et));
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    accH[kd][q] = mul2(accH[kd][q], f);
                    accL[kd][q] = mul2(accL[kd][q], f);
                }
                Erun[kd] = Et;
            }
        }
        {
            const float2 wq = df_split(w.hQ, Erun[0] - 1023);
            const float2 wm = df_split(w.hM, Erun[1] - 1023);
            const float2 wg = df_split(w.hG, Erun[2] - 1023);
            Trow[0] = make_float4(2.0f * sd.x, 2.0f * sd.y, wq.x, wq.y);
            Trow[1] = make_float4(wm.x, wm.y, wg.x, wg.y);
        }
        __syncthreads();
        if (bact) {
            // rows in groups of eight, the accumulators renormalised after each; the
            // twelve multiply-adds of a row as six pairs (columns 4 qi, 4 qi + 1 and
            // 4 qi + 2, 4 qi + 3 in the two lanes)
            const int aslot = 1 + (qi > 0 ? qi : 1);
            for (int m0 = mlo; m0 < mhi; m0 += 8) {
                const int m1 = min(mhi, m0 + 8);
                const float4* Tm = sT + m0 * rs4;
                for (int m = m0; m < m1; ++m, Tm += rs4) {
                    const float4 h01 = Tm[0];
                    const float4 h23 = Tm[1];
                    const float4 an = Tm[aslot];
                    const float2 s2 = make_float2(h01.x, h01.y);
                    // (T_4qi, T_4qi+1): the anchors, or (T_0, T_1) = (1, s)
                    const float2 aH = qi > 0 ? make_float2(an.x, an.y) : make_float2(1.0f, 0.5f * h01.x);
                    const float2 aL = qi > 0 ? make_float2(an.z, an.w) : make_float2(0.0f, 0.5f * h01.y);
                    const float2 t0 = make_float2(aH.x, aL.x), t1 = make_float2(aH.y, aL.y);
                    const float2 t2 = df_mulsub(s2, t1, t0);
                    const float2 t3 = df_mulsub_nr(s2, t2, t1);  // (a product operand only)
                    const float2 bH = make_float2(t2.x, t3.x), bL = make_float2(t2.y, t3.y);
                    const float2 naH = neg2(aH), nbH = neg2(bH);
                    const float2 wH[3] = {bcast2(h01.z), bcast2(h23.x), bcast2(h23.z)};
                    const float2 wL[3] = {bcast2(h01.w), bcast2(h23.y), bcast2(h23.w)};
#pragma unroll
                    for (int kd = 0; kd < 3; ++kd) {
                        df_fma2(accH[kd][0], accL[kd][0], wH[kd], wL[kd], aH, aL, naH);
                        df_fma2(accH[kd][1], accL[kd][1], wH[kd], wL[kd], bH, bL, nbH);
                    }
                }
#pragma unroll
                for (int kd = 0; kd < 3; ++kd)
#pragma unroll
                    for (int q = 0; q < 2; ++q) df_renorm2(accH[kd][q], accL[kd][q]);
            }
        }
        __syncthreads();
    }

    // combine the groups (double-float, at the common running scale) in a fixed
    // order, widen to FP64 and write this block's split; T_0 enters as 1/2
    float2* red = reinterpret_cast<float2*>(smem);  // [G][3][N]
    if (bact) {
#pragma unroll
        for (int kd = 0; kd < 3; ++kd)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = 4 * qi + q;
                if (j < N) {
                    const float2 hh = accH[kd][q >> 1], ll = accL[kd][q >> 1];
                    float2 v = (q & 1) ? make_float2(hh.y, ll.y) : make_float2(hh.x, ll.x);
                    if (j == 0) v = make_float2(0.5f * v.x, 0.5f * v.y);
                    red[((size_t)g * 3 + kd) * N + j] = v;
                }
            }
    }
    __syncthreads();
    double* out = A.Vpart + ((size_t)rt * A.KS + ks) * 3 * (size_t)N;
    for (int idx = tid; idx < 3 * N; idx += BT) {
        float2 v = red[idx];
        for (int gg = 1; gg < G; ++gg) v = df_add(v, red[(size_t)gg * 3 * N + idx]);
        const int kd = idx / N;
        const int E = kd == 0 ? Erun[0] : kd == 1 ? Erun[1] : Erun[2];
        out[idx] = df_widen(v.x, E) + df_widen(v.y, E);
    }
}

// factors per radial node in the batched tile (the FP64 ones of the single tile)
constexpr int kRadFactorsBatched = 8;

// Row layout of the batched tile: T_0 .. T_N-1 per triple (N + 1 pairs).
__host__ __device__ inline int row_len_for(int N) { return N + 1; }

__host__ __device__ inline int groups_for(int N, int BT) {
    const int nact = N < BT ? N : BT;
    return BT / nact;
}

__host__ __device__ inline size_t tile_doubles(bool full, int N, int BT) {
    if (!full) return 0;
    const size_t t = (size_t)BT * (size_t)row_len_for(N);
    const size_t red = (size_t)groups_for(N, BT) * 3u * (size_t)N;
    return t > red ? t : red;
}

__host__ __device__ inline size_t smem_doubles(bool full, int N, int BT) {
    // tile rows, 3 BT weights as double-float pairs, 2 N coefficients, 4 boundary
    // sums, 3 x 8 per-warp exponent maxima, the factors of a group of radial nodes
    return tile_doubles(full, N, BT) + 3u * (size_t)BT + 2u * (size_t)N + 4u + 12u +
           (size_t)kRadGroup * kRadFactorsBatched;
}

// One work item of the persistent batched kernel: row rt, radial split ks of the
// problem in A.  The shared-memory row of a triple holds T_0 .. T_N-1 (T_0 as 1/2)
// as double-float pairs; phase-B thread j accumulates column j.  smem holds
// smem_doubles(FULL, N, BT) doubles.
template <int BT, int NJ, bool FULL>
__device__ __forceinline__ void triple_tile_batched(const TripleArgs& A, const int rt, const int ks, double* smem) {
    const Consts& c = A.c;
    const int N = c.N;
    const int ldT = row_len_for(N);
    double* sT = smem;
    float2* sT2 = reinterpret_cast<float2*>(smem);  // rows T_0 .. T_N-1 as double-float pairs
    float2* sh2 = reinterpret_cast<float2*>(smem + tile_doubles(FULL, N, BT));  // [3][BT] weight pairs
    double* sa = smem + tile_doubles(FULL, N, BT) + 3 * BT;
    double* sb = sa + N;
    double* sbnd = sb + N;  // ln Z(s=1), ln G(s=1), ln Z(s=-1), ln G(s=-1) (table path)
    int* sex = reinterpret_cast<int*>(sbnd + 4);  // [3][8] per-warp maxima of the weights' exponents
    double* srad = sbnd + 16;                     // [kRadGroup][kRadFactorsBatched] radial-node factors
    constexpr int WARPS = BT / 32;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;

    // a (NZ) and b (NG) zero-padded to N = max(NZ, NG): one recurrence serves both series
    for (int j = tid; j < N; j += BT) {
        sa[j] = j < c.NZ ? A.coef[j] : 0.0;
        sb[j] = j < c.NG ? A.coef[c.NZ + j] : 0.0;
    }
    const Row row = A.rows[rt];
    const bool gluon = (row.flags & kRowGluon) != 0;
    const bool ghost = (row.flags & kRowGhost) != 0;
    const int k0 = ks * A.KB;
    const int k1 = min(c.nr, k0 + A.KB);
    const int nch = A.nch;
    const int nunits = k1 > k0 ? (k1 - k0) * nch : 0;

    // phase-B mapping: NG groups of nact threads, thread owns the columns
    // j = jb + jj*nact
    const int ncol = N;
    const int nact = ncol < BT ? ncol : BT;
    const int NG = BT / nact;
    const int g = tid / nact;
    const int jb = tid - g * nact;
    const bool bact = g < NG;
    const int mlo = (g * BT) / NG;
    const int mhi = ((g + 1) * BT) / NG;
    int colj[NJ];
#pragma unroll
    for (int jj = 0; jj < NJ; ++jj) {
        const int cc = jb + jj * nact;
        colj[jj] = cc < N ? cc : N;  // j >= N: inactive
    }

    double acc[3][NJ];
#pragma unroll
    for (int jj = 0; jj < NJ; ++jj) acc[0][jj] = acc[1][jj] = acc[2][jj] = 0.0;
    static_assert(WARPS <= 8, "per-warp exponent maxima hold 8 warps");

    const float ith_scale = (float)c.sM * (float)(1.0 / kPi);  // theta -> interval index
    // the series at s = +-1 from the table's end-point record
    if (A.stab && tid < 4) sbnd[tid] = reinterpret_cast<const double*>(A.stab + kSeriesM)[tid];
    __syncthreads();

    // (x, y) factors of the integrands, formed once per radial node instead of per
    // triple: z = d + b2 sigma with d = (sqrt x - sqrt y)^2, b2 = 4 sqrt(xy);
    // K = W_k y G(y) (hM = K w s4 G(z)/z, hG = K w s4 Z(z)/z^2); the quartic of the
    // gluon-loop kernel times W_k W(y)/2 (hQ = w s2 W(z)/z^2 sum_i kQ_i sigma^i).
    // A group of kRadGroup nodes spans whole tiles: kRadGroup nch is a multiple of WARPS.
    const int group_units = kRadGroup * nch;
    for (int base = 0; base < nunits; base += WARPS) {
        if (base % group_units == 0) {
            __syncthreads();  // the previous group's factors are no longer read
            if (warp == 0) {
                const int kq = k0 + base / nch + lane;
                if (kq < k1) {
                    const Rad rd = A.rad[rad_offset(c, rt) + kq];
                    const YTab yt = A.ytab[rad_offset(c, rt) + kq];
                    const double d0 = row.sx - rd.sy;
                    const double d = d0 * d0;
                    const double b = 2.0 * row.sx * rd.sy;
                    double* f = srad + lane * kRadFactorsBatched;
                    f[0] = d;
                    f[1] = 2.0 * b;
                    f[2] = rd.W * yt.yG;
                    const double dd = d * d, db = d * b, bb = b * b;
                    const double h = 0.5 * rd.W * yt.Wy;
                    f[3] = h * (7.5 * dd);
                    f[4] = h * -(48.0 * dd + 18.0 * db + 12.0 * bb);
                    f[5] = h * (48.0 * dd - 48.0 * db - 38.0 * bb);
                    f[6] = h * (96.0 * db + 64.0 * bb);
                    f[7] = h * (16.0 * bb);
                }
            }
            __syncthreads();
        }
        const int u = base + warp;
        double hQ = 0.0, hM = 0.0, hG = 0.0;
        float2* Trow = sT2 + (size_t)tid * ldT;
        bool live = false;
        int k = 0, ch = 0;
        if (u < nunits) {
            const int kk = u / nch;
            ch = u - kk * nch;
            k = k0 + kk;
            const int l = ch * 32 + lane;
            if (l < c.na) {
                live = true;
                const double* f = srad + (kk % kRadGroup) * kRadFactorsBatched;
                const Ang an = A.ang[l];
                const double z = fma(f[1], an.sig, f[0]);
                const LnRcp lr = ln_rcp(z);
                const double lz = lr.ln;
                // s(z), clamped to [-1, 1] for z outside [eps2, lambda2] (inside, it can
                // leave the interval only by a rounding)
                double s = (lz - c.L0) * c.invL1;
                const double iz = lr.rcp;
                const double iz2 = iz * iz;
                double Zz = 0.0, Gz = 0.0, Wz = 0.0;  // Z(z), G(z), W(z) = G(z)^p Z(z)^q
                // z > 0: the comparisons with eps2, lambda2 on the bit patterns
                const long long zb = __double_as_longlong(z);
                const bool beyond = zb < __double_as_longlong(c.eps2) || zb > __double_as_longlong(c.lam2);
                const bool outside = c.extrap == 0 && beyond;
                if (beyond) s = fmin(1.0, fmax(-1.0, s));
                if (A.stab && !outside) {
                    // Z(z), G(z), W(z) from the table: the interval by arccos in
                    // FP32 (FP32 s from the bits of s, truncated: the interval only),
                    // the polynomials in u = (s - mid) / half in double-float
                    const float sf = fminf(1.0f, fmaxf(-1.0f, df_split(s, 0).x));
                    int it = (int)(acosf(sf) * ith_scale);
                    it = min(max(it, 0), c.sM - 1);
                    const SeriesRec* Rr = A.stab + it;
                    const double2 mh = __ldg(reinterpret_cast<const double2*>(Rr));
                    series_eval(Rr, df_split((s - mh.x) * mh.y, 0), ghost || gluon, gluon, Zz, Gz, Wz);
                } else {
                    double lg, lzz;
                    if (A.stab) {
                        // outside [eps2, lambda2]: the series at s = +-1 (block sums)
                        lzz = s > 0.0 ? sbnd[0] : sbnd[2];
                        lg = s > 0.0 ? sbnd[1] : sbnd[3];
                    } else {
                        lg = 0.5 * sb[0];
                        lzz = 0.5 * sa[0];
                        if (N > 1) {
                            lg = fma(sb[1], s, lg);
                            lzz = fma(sa[1], s, lzz);
                        }
                        double t0 = 1.0, t1 = s;
                        const double s2x = 2.0 * s;
                        for (int j = 2; j < N; ++j) {
                            const double t2 = fma(s2x, t1, -t0);
                            t0 = t1;
                            t1 = t2;
                            lg = fma(sb[j], t2, lg);
                            lzz = fma(sa[j], t2, lzz);
                            if (FULL) Trow[j] = df_split(t2, 0);
                        }
                    }
                    if (outside) {
                        if (z < c.eps2) {
                            const double r = lz - c.ln_eps2;
                            lg = fma(-c.kappa, r, lg);
                            lzz = fma(2.0 * c.kappa, r, lzz);
                        } else {
                            const double L = log1p(c.omega * (lz - c.ln_lam2));
                            lg = fma(c.delta, L, lg);
                            lzz = fma(c.gam, L, lzz);
                        }
                    }
                    if (ghost) Zz = exp(lzz);
                    if (gluon) {
                        Gz = exp(lg);
                        Wz = exp(c.pG * lg + c.qZ * lzz);
                    }
                }
                if (FULL) {
                    const float2 fs = df_split(s, 0);
                    Trow[0] = make_float2(0.5f, 0.0f);  // T_0 enters as 1/2
                    if (N > 1) Trow[1] = fs;
                    if (A.stab) {
                        // T_4i, T_4i+1 by the double-float recurrence of stride 4 (see
                        // below), T_4i+2 and T_4i+3 by two double-float steps (the direct
                        // path stored all)
                        const double T2 = fma(2.0 * s, s, -1.0);
                        const double T3 = fma(2.0 * s, T2, -s);
                        const double T4 = fma(2.0 * T2, T2, -1.0);
                        const float2 c4 = df_split(2.0 * T4, 0);
                        const float2 s2 = make_float2(2.0f * fs.x, 2.0f * fs.y);
                        float2 a0 = df_split(T4, 0), a1 = make_float2(1.0f, 0.0f);  // T_(4i-4), T_4i
                        float2 b0 = df_split(T3, 0), b1 = fs;                       // T_(4i-3), T_(4i+1)
                        for (int j0 = 0; j0 < N; j0 += 4) {
                            if (j0 > 0) {
                                Trow[j0] = a1;
                                if (j0 + 1 < N) Trow[j0 + 1] = b1;
                            }
                            if (j0 + 2 < N) {
                                const float2 t2 = df_mulsub(s2, b1, a1);
                                Trow[j0 + 2] = t2;
                                if (j0 + 3 < N) Trow[j0 + 3] = df_mulsub(s2, t2, b1);
                            }
                            const float2 an4 = df_mulsub(c4, a1, a0);
                            a0 = a1;
                            a1 = an4;
                            const float2 bn = df_mulsub(c4, b1, b0);
                            b0 = b1;
                            b1 = bn;
                        }
                    }
                }
                const double Kw = f[2] * an.ws4;
                if (ghost) hG = Kw * Zz * iz2;
                if (gluon) {
                    const double sg = an.sig;
                    const double num = fma(sg, fma(sg, fma(sg, fma(sg, f[7], f[6]), f[5]), f[4]), f[3]);
                    hQ = an.ws2 * iz2 * Wz * num;
                    hM = Kw * iz * Gz;
                }
            }
        }
        if (FULL && !live) {
            for (int j = 0; j < ldT; ++j) Trow[j] = make_float2(0.0f, 0.0f);
        }
        // angular sums over the warp's 32 nodes (same radial node for the whole
        // warp) of (hQ, hM, hG) by halving exchanges, 6 FP64 additions per lane:
        // lanes 0-15 go on with (hQ, hM), lanes 16-31 with (hG, 0); then lanes with
        // bit 3 set with the second of the two; then three butterfly steps.  The
        // sums end in lanes 0 (hQ), 8 (hM) and 16 (hG).
        {
            const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0;
            const double k0 = (h16 ? hG : hQ) + __shfl_xor_sync(kFullMask, h16 ? hQ : hG, 16);
            const double k1 = (h16 ? 0.0 : hM) + __shfl_xor_sync(kFullMask, h16 ? hM : 0.0, 16);
            double v = (h8 ? k1 : k0) + __shfl_xor_sync(kFullMask, h8 ? k0 : k1, 8);
            v += __shfl_xor_sync(kFullMask, v, 4);
            v += __shfl_xor_sync(kFullMask, v, 2);
            v += __shfl_xor_sync(kFullMask, v, 1);
            if (u < nunits && (lane & 7) == 0 && lane < 24) {
                double* up = A.Upart + (((size_t)rt * c.nr + k) * nch + ch) * 3;
                up[lane >> 3] = v;
            }
        }
        if (FULL) {
            // per-tile power-of-two scale of each weight kind: the largest exponent
            {
                const unsigned eq = ((unsigned)__double2hiint(hQ) >> 20) & 0x7ffu;
                const unsigned em = ((unsigned)__double2hiint(hM) >> 20) & 0x7ffu;
                const unsigned eg = ((unsigned)__double2hiint(hG) >> 20) & 0x7ffu;
                const unsigned mq = __reduce_max_sync(kFullMask, eq);
                const unsigned mm = __reduce_max_sync(kFullMask, em);
                const unsigned mg = __reduce_max_sync(kFullMask, eg);
                if (lane == 0) {
                    sex[warp] = (int)mq;
                    sex[8 + warp] = (int)mm;
                    sex[16 + warp] = (int)mg;
                }
            }
            __syncthreads();
            int Eq = sex[0], Em = sex[8], Eg = sex[16];
#pragma unroll
            for (int w = 1; w < WARPS; ++w) {
                Eq = max(Eq, sex[w]);
                Em = max(Em, sex[8 + w]);
                Eg = max(Eg, sex[16 + w]);
            }
            // weights w 2^-(E - 1023): the largest lands in [1, 2)
            sh2[tid] = df_split(hQ, Eq - 1023);
            sh2[BT + tid] = df_split(hM, Em - 1023);
            sh2[2 * BT + tid] = df_split(hG, Eg - 1023);
            __syncthreads();
            if (bact) {
                float2 ca[3][NJ];
#pragma unroll
                for (int jj = 0; jj < NJ; ++jj) ca[0][jj] = ca[1][jj] = ca[2][jj] = make_float2(0.0f, 0.0f);
                for (int m0 = mlo; m0 < mhi; m0 += 8) {
                    const int m1 = min(mhi, m0 + 8);
                    for (int m = m0; m < m1; ++m) {
                        const float2 q = sh2[m];
                        const float2 mm = sh2[BT + m];
                        const float2 gg = sh2[2 * BT + m];
                        const float2* Tm = sT2 + (size_t)m * ldT;
#pragma unroll
                        for (int jj = 0; jj < NJ; ++jj) {
                            if (colj[jj] < N) {
                                const float2 t = Tm[colj[jj]];
                                df_fma(ca[0][jj], q, t);
                                df_fma(ca[1][jj], mm, t);
                                df_fma(ca[2][jj], gg, t);
                            }
                        }
                    }
#pragma unroll
                    for (int jj = 0; jj < NJ; ++jj) {
                        df_renorm(ca[0][jj]);
                        df_renorm(ca[1][jj]);
                        df_renorm(ca[2][jj]);
                    }
                }
                // tile sums into the FP64 accumulators, scaled back by 2^(E - 1023)
#pragma unroll
                for (int jj = 0; jj < NJ; ++jj) {
                    acc[0][jj] += df_widen(ca[0][jj].x, Eq) + df_widen(ca[0][jj].y, Eq);
                    acc[1][jj] += df_widen(ca[1][jj].x, Em) + df_widen(ca[1][jj].y, Em);
                    acc[2][jj] += df_widen(ca[2][jj].x, Eg) + df_widen(ca[2][jj].y, Eg);
                }
            }
            __syncthreads();
        }
    }

    if (FULL) {
        // combine the groups in a fixed order and write this block's split
        double* red = sT;  // [NG][3][N]
        if (bact) {
#pragma unroll
            for (int jj = 0; jj < NJ; ++jj) {
                const int j = colj[jj];
                if (j < N) {
                    red[(g * 3 + 0) * N + j] = acc[0][jj];
                    red[(g * 3 + 1) * N + j] = acc[1][jj];
                    red[(g * 3 + 2) * N + j] = acc[2][jj];
                }
            }
        }
        __syncthreads();
        double* out = A.Vpart + ((size_t)rt * A.KS + ks) * 3 * (size_t)N;
        for (int idx = tid; idx < 3 * N; idx += BT) {
            double s = 0.0;
            for (int gg = 0; gg < NG; ++gg) s += red[(size_t)gg * 3 * N + idx];
            out[idx] = s;
        }
    }
}

// Newton-matrix mode: blocks of BT threads; with BT = 128 six blocks per SM (at
// most 80 registers a thread)
#ifndef DSE_TRIPLE_MIN_BLOCKS
#define DSE_TRIPLE_MIN_BLOCKS 6
#endif
template <int BT>
__global__ void __launch_bounds__(BT, BT == 128 ? DSE_TRIPLE_MIN_BLOCKS : 8) k_triple(const __grid_constant__ TripleArgs A) {
    extern __shared__ __align__(16) double smem[];
    triple_tile_full<BT>(A, blockIdx.y, blockIdx.x, smem);
}

// Residual mode: blocks of BT threads
template <int BT>
__global__ void __launch_bounds__(BT) k_triple_res(const __grid_constant__ TripleArgs A) {
    extern __shared__ __align__(16) double smem[];
    triple_tile_residual<BT>(A, blockIdx.y, blockIdx.x, smem);
}

// Persistent form for a batch of independent problems: each block takes work
// items (problem, row, radial split) from a global counter in the order of the
// item list (longest first) until the list is exhausted; items of converged
// problems are skipped.
template <int BT, int NJ, bool FULL>
__global__ void __launch_bounds__(BT) k_triple_batched(const BatchProblem* __restrict__ P,
                                                       const BatchItem* __restrict__ items, int n_items,
                                                       int* __restrict__ counter,
                                                       const double* __restrict__ coef_base) {
    extern __shared__ __align__(16) double smem[];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();  // also orders the previous item's shared-memory use before this one
        const int it = s_item;
        __syncthreads();
        if (it >= n_items) break;
        const BatchItem w = items[it];
        if (!P[w.b].active) continue;
        TripleArgs A = P[w.b].t;
        A.coef = coef_base + P[w.b].coef_off;
        triple_tile_batched<BT, NJ, FULL>(A, w.rt, w.ks, smem);
    }
}

template <int BT>
cudaError_t launch_full(const TripleArgs& a, cudaStream_t s) {
    const size_t smem = smem_full_doubles(a.c.N, BT, a.KB) * sizeof(double);
    const dim3 grid(a.KS, a.Rt);
    cudaError_t e = cudaFuncSetAttribute(k_triple<BT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_triple<BT><<<grid, BT, smem, s>>>(a);
    return cudaGetLastError();
}

template <int BT>
cudaError_t launch_res(const TripleArgs& a, cudaStream_t s) {
    const size_t smem = smem_res_doubles(a.c.N, a.KB) * sizeof(double);
    const dim3 grid(a.KS, a.Rt);
    cudaError_t e = cudaFuncSetAttribute(k_triple_res<BT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_triple_res<BT><<<grid, BT, smem, s>>>(a);
    return cudaGetLastError();
}

// resident blocks per SM (with the radial-factor store of two nodes per block,
// the fewest the split uses)
template <int BT>
int occupancy_full(int N) {
    const size_t smem = smem_full_doubles(N, BT, 2) * sizeof(double);
    int nb = 0;
    cudaFuncSetAttribute(k_triple<BT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_triple<BT>, BT, smem);
    return e == cudaSuccess ? nb : 0;
}

int occupancy_res(int N) {
    const size_t smem = smem_res_doubles(N, 2) * sizeof(double);
    int nb = 0;
    cudaFuncSetAttribute(k_triple_res<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_triple_res<128>, 128, smem);
    return e == cudaSuccess ? nb : 0;
}

}  // namespace

int triple_block_threads(int N) { return block_threads_for(N); }

size_t triple_smem_bytes(bool full, int N, int KB) {
    return (full ? smem_full_doubles(N, block_threads_for(N), KB) : smem_res_doubles(N, KB)) * sizeof(double);
}

int triple_max_blocks_per_sm(bool full, int N) {
    if (!full) return occupancy_res(N);
    return block_threads_for(N) == 128 ? occupancy_full<128>(N) : occupancy_full<64>(N);
}

namespace {
template <int BT, bool FULL>
cudaError_t launch_batched_bt(const BatchProblem* P, const BatchItem* items, int n_items, int* counter,
                              const double* coef_base, int maxN, int grid, cudaStream_t s) {
    const size_t smem = smem_doubles(FULL, maxN, BT) * sizeof(double);
    const int nj = (maxN + BT - 1) / BT;
    // the shared-memory limit was set by triple_batched_blocks_per_sm (no attribute
    // change here: this launch may be captured into a graph)
#define DSE_LAUNCH_TB(NJ) k_triple_batched<BT, NJ, FULL><<<grid, BT, smem, s>>>(P, items, n_items, counter, coef_base);
    if (nj <= 1) { DSE_LAUNCH_TB(1) }
    else if (nj <= 2) { DSE_LAUNCH_TB(2) }
    else if (nj <= 4) { DSE_LAUNCH_TB(4) }
    else return cudaErrorInvalidValue;
#undef DSE_LAUNCH_TB
    return cudaGetLastError();
}

template <int BT, bool FULL>
int batched_occupancy_bt(int maxN) {
    const size_t smem = smem_doubles(FULL, maxN, BT) * sizeof(double);
    const int nj = (maxN + BT - 1) / BT;
    int nb = 0;
    cudaError_t e;
    if (nj <= 1) {
        cudaFuncSetAttribute(k_triple_batched<BT, 1, FULL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_triple_batched<BT, 1, FULL>, BT, smem);
    } else if (nj <= 2) {
        cudaFuncSetAttribute(k_triple_batched<BT, 2, FULL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_triple_batched<BT, 2, FULL>, BT, smem);
    } else {
        cudaFuncSetAttribute(k_triple_batched<BT, 4, FULL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_triple_batched<BT, 4, FULL>, BT, smem);
    }
    return e == cudaSuccess ? nb : 0;
}
}  // namespace

cudaError_t launch_triple_batched(bool full, const BatchProblem* P, const BatchItem* items, int n_items,
                                  int* counter, const double* coef_base, int maxN, int grid, cudaStream_t s) {
    if (n_items <= 0 || grid <= 0) return cudaSuccess;
    if (block_threads_for(maxN) == 128)
        return full ? launch_batched_bt<128, true>(P, items, n_items, counter, coef_base, maxN, grid, s)
                    : launch_batched_bt<128, false>(P, items, n_items, counter, coef_base, maxN, grid, s);
    return full ? launch_batched_bt<64, true>(P, items, n_items, counter, coef_base, maxN, grid, s)
                : launch_batched_bt<64, false>(P, items, n_items, counter, coef_base, maxN, grid, s);
}

int triple_batched_blocks_per_sm(bool full, int maxN) {
    if (block_threads_for(maxN) == 128)
        return full ? batched_occupancy_bt<128, true>(maxN) : batched_occupancy_bt<128, false>(maxN);
    return full ? batched_occupancy_bt<64, true>(maxN) : batched_occupancy_bt<64, false>(maxN);
}

cudaError_t launch_triple(bool full, const TripleArgs& a, cudaStream_t s) {
    if (a.KS <= 0 || a.Rt <= 0) return cudaSuccess;
    if (!full) return launch_res<128>(a, s);
    return block_threads_for(a.c.N) == 128 ? launch_full<128>(a, s) : launch_full<64>(a, s);
}

}  // namespace dse
