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
#include "dse_lntab.cuh"

namespace dse {

namespace {

constexpr unsigned kFullMask = 0xffffffffu;
constexpr double kPi = 3.14159265358979323846264338327950288;

__host__ __device__ inline int block_threads_for(int N) { return N <= 96 ? 128 : 64; }

// ---- ln z and 1/z (table-driven, Tang 1990) ----
// z = 2^e m with m in [1, 2); for the leading 7 fraction bits j of m, c_j =
// 1 + (j + 1/2)/128, inv_j = 1/c_j rounded to FP64 and L_j = -ln(inv_j) as a
// double-double (dse_lntab.cuh, written by gen_lntab.py with 60-digit arithmetic).  With r = m inv_j - 1
// (one FMA, |r| < 2^-7.9):
//   ln z = e ln2 + L_j + ln(1 + r),  ln(1 + r) = r - r^2/2 + r^3/3 (FP64)
//          - r^4 (1/4 - r/5 + r^2/6 - r^3/7) (FP32, below 2.4e-10);
//   1/z = 2^-e inv_j / (1 + r),  1/(1 + r) = ((1 - r) + r^2) - r^3 (FP64) + r^4 (1 - r + r^2) (FP32).
// ln2 = ln2_hi + ln2_lo with ln2_hi holding 42 significant bits, so e ln2_hi is exact.
// Accuracy (emulated against 40-digit arithmetic over z in [1e-14, 1e8]): ln z within
// 2 units of 2^-53 max(1, |ln z|), 1/z within 4 units in the last place.  Zero,
// subnormal, very large, infinite and NaN arguments take the library routines.
constexpr int kLnTab = 128;  // g_lntab: inv_j, L_j hi, L_j lo (kLnTab each), ln2_hi, ln2_lo

struct LnRcp { double ln, rcp; };

__device__ __forceinline__ LnRcp ln_rcp(double z) {
    LnRcp o;
    if (!(z >= 0x1p-1020 && z <= 0x1p+1020)) {
        o.ln = log(z);
        o.rcp = 1.0 / z;
        return o;
    }
    const int hz = __double2hiint(z);
    const int e = ((hz >> 20) & 0x7ff) - 1023;
    const int j = (hz >> 13) & (kLnTab - 1);
    const double m = __hiloint2double((hz & 0x000fffff) | 0x3ff00000, __double2loint(z));
    const double inv = __ldg(&g_lntab[j]);
    const double Lh = __ldg(&g_lntab[kLnTab + j]), Ll = __ldg(&g_lntab[2 * kLnTab + j]);
    const double ln2h = __ldg(&g_lntab[3 * kLnTab]), ln2l = __ldg(&g_lntab[3 * kLnTab + 1]);
    const double r = fma(m, inv, -1.0);
    const double r2 = r * r;
    const double r3 = r2 * r;
    const float rf = df_split(r, 0).x;  // r to FP32 precision (truncated)
    const float r4f = (rf * rf) * (rf * rf);
    const float tl = r4f * fmaf(fmaf(fmaf(-1.0f / 7.0f, rf, 1.0f / 6.0f), rf, -0.2f), rf, 0.25f);
    const float tq = r4f * fmaf(rf, rf - 1.0f, 1.0f);
    // e as a double without a conversion instruction: 1.5 2^52 + (e + 2^31) - (1.5 2^52 + 2^31)
    const double ed = __hiloint2double(0x43380000, (int)((unsigned)e ^ 0x80000000u)) - 6755401588539392.0;
    const double lead = fma(r3, 1.0 / 3.0, fma(r2, -0.5, r));
    const double hi = fma(ed, ln2h, Lh);
    const double lo = fma(ed, ln2l, Ll);
    o.ln = hi + ((lead - df_widen(tl, 1023)) + lo);
    const double q = (((1.0 - r) + r2) - r3) + df_widen(tq, 1023);
    o.rcp = (q * inv) * __hiloint2double((1023 - e) << 20, 0);
    return o;
}

// The shared-memory row of a triple holds 2s and the anchors T_4i, T_4i+1
// (i < nq = ceil(N/4)) as double-float pairs; phase B forms T_4i+2 = 2s T_4i+1 - T_4i
// and T_4i+3 = 2s T_4i+2 - T_4i+1 from them.  Its 4 nq derivative columns c map to
// j = 4 (c mod nq) + c div nq, so that a warp's threads share c div nq (the same
// number of recurrence steps) when nq is a multiple of 16.
// With AR false (full rows) the row holds T_0 .. T_N-1 (T_0 as 1/2) and column c
// is j = c: twice the shared memory, no recurrence steps in phase B.
__host__ __device__ inline int anchors_for(int N) { return (N + 3) / 4; }
__host__ __device__ inline int row_len_for(int N, bool ar) {
    if (!ar) return N + 1;
    const int l = 1 + 2 * anchors_for(N);
    return l | 1;  // odd: conflict-free rows
}

__host__ __device__ inline int ncols_for(int N, bool ar) { return ar ? 4 * anchors_for(N) : N; }

__host__ __device__ inline int groups_for(int N, int BT, bool ar) {
    const int nc = ncols_for(N, ar);
    const int nact = nc < BT ? nc : BT;
    return BT / nact;
}

__host__ __device__ inline size_t tile_doubles(bool full, int N, int BT, bool ar) {
    if (!full) return 0;
    const size_t t = (size_t)BT * (size_t)row_len_for(N, ar);
    const size_t red = (size_t)groups_for(N, BT, ar) * 3u * (size_t)N;
    return t > red ? t : red;
}

// Row layout of each kernel: the single-problem kernel keeps anchor rows (more
// blocks per SM); the persistent batched kernel, limited by its registers, full rows.
constexpr bool kAnchorRowsSingle = true;
constexpr bool kAnchorRowsBatched = false;

// Radial nodes whose per-node factors are formed together (by one warp) and
// kept in shared memory, and the factors per node.
constexpr int kRadGroup = 32;
constexpr int kRadFactors = 8;

__host__ __device__ inline size_t smem_doubles(bool full, int N, int BT, bool ar) {
    // tile rows, 3 BT weights as double-float pairs, 2 N coefficients, 4 boundary
    // sums, 3 x 8 per-warp exponent maxima, the factors of a group of radial nodes
    return tile_doubles(full, N, BT, ar) + 3u * (size_t)BT + 2u * (size_t)N + 4u + 12u +
           (size_t)kRadGroup * kRadFactors;
}

// One block's work: row rt, radial split ks of the problem in A.  smem holds
// smem_doubles(FULL, N, BT, AR) doubles.
template <int BT, int NJ, bool FULL, bool AR>
__device__ __forceinline__ void triple_tile(const TripleArgs& A, const int rt, const int ks, double* smem) {
    const Consts& c = A.c;
    const int N = c.N;
    const int nq = anchors_for(N);
    const int ldT = row_len_for(N, AR);
    double* sT = smem;
    float2* sT2 = reinterpret_cast<float2*>(smem);  // rows [2s][T_4i][T_4i+1] as double-float pairs
    float2* sh2 = reinterpret_cast<float2*>(smem + tile_doubles(FULL, N, BT, AR));  // [3][BT] weight pairs
    double* sa = smem + tile_doubles(FULL, N, BT, AR) + 3 * BT;
    double* sb = sa + N;
    double* sbnd = sb + N;  // ln Z(s=1), ln G(s=1), ln Z(s=-1), ln G(s=-1) (table path)
    int* sex = reinterpret_cast<int*>(sbnd + 4);  // [3][8] per-warp maxima of the weights' exponents
    double* srad = sbnd + 16;                     // [kRadGroup][kRadFactors] radial-node factors
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
    // c = jb + jj*nact of 4 nq: T_j with j = 4 (c mod nq) + c div nq
    const int ncol = ncols_for(N, AR);
    const int nact = ncol < BT ? ncol : BT;
    const int NG = BT / nact;
    const int g = tid / nact;
    const int jb = tid - g * nact;
    const bool bact = g < NG;
    const int mlo = (g * BT) / NG;
    const int mhi = ((g + 1) * BT) / NG;
    int colj[NJ], coli[NJ], colr[NJ];
#pragma unroll
    for (int jj = 0; jj < NJ; ++jj) {
        const int cc = jb + jj * nact;
        colr[jj] = AR ? cc / nq : 0;
        coli[jj] = AR ? cc - colr[jj] * nq : 0;
        if (AR) colj[jj] = cc < ncol ? 4 * coli[jj] + colr[jj] : N;  // j >= N: inactive
        else colj[jj] = cc < N ? cc : N;
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
                    double* f = srad + lane * kRadFactors;
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
                const double* f = srad + (kk % kRadGroup) * kRadFactors;
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
                    // FP32, the polynomials in u = (s - mid) / half in FP64 (Horner)
                    // (FP32 s from the bits of s, truncated: the interval only)
                    const float sf = fminf(1.0f, fmaxf(-1.0f, df_split(s, 0).x));
                    int it = (int)(acosf(sf) * ith_scale);
                    it = min(max(it, 0), c.sM - 1);
                    const SeriesRec* R = A.stab + it;
                    const double2 mh = __ldg(reinterpret_cast<const double2*>(R));
                    const double uu = (s - mh.x) * mh.y;
                    // Horner: the tail (degree kSeriesLead .. kSeriesP) in double-float,
                    // the leading coefficients in FP64
                    const float2 uf = df_split(uu, 0);
                    if (ghost || gluon) {
                        const float4 top = __ldg(&R->et[kSeriesTail - 1]);
                        float2 tz = make_float2(top.x, top.y), tg = make_float2(top.z, top.w);
#pragma unroll
                        for (int kq = kSeriesTail - 2; kq >= 0; --kq) {
                            const float4 ck = __ldg(&R->et[kq]);
                            tz = df_muladd(tz, uf, make_float2(ck.x, ck.y));
                            tg = df_muladd(tg, uf, make_float2(ck.z, ck.w));
                        }
                        double ez = df_widen(tz.x, 1023) + df_widen(tz.y, 1023);
                        double eg = df_widen(tg.x, 1023) + df_widen(tg.y, 1023);
#pragma unroll
                        for (int kq = kSeriesLead - 1; kq >= 0; --kq) {
                            const double2 ck = __ldg(&R->e[kq]);
                            ez = fma(ez, uu, ck.x);
                            eg = fma(eg, uu, ck.y);
                        }
                        Zz = ez;
                        Gz = eg;
                    }
                    if (gluon) {
                        float2 tw = __ldg(&R->wt[kSeriesTail - 1]);
#pragma unroll
                        for (int kq = kSeriesTail - 2; kq >= 0; --kq) tw = df_muladd(tw, uf, __ldg(&R->wt[kq]));
                        double ew = df_widen(tw.x, 1023) + df_widen(tw.y, 1023);
#pragma unroll
                        for (int kq = kSeriesLead - 1; kq >= 0; --kq) ew = fma(ew, uu, __ldg(&R->w[kq]));
                        Wz = ew;
                    }
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
                            if (FULL && AR && (j & 3) < 2) Trow[1 + (j & 1) * nq + (j >> 2)] = df_split(t2, 0);
                            if (FULL && !AR) Trow[j] = df_split(t2, 0);
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
                if (FULL && !AR) {
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
                if (FULL && AR) {
                    const float2 fs = df_split(s, 0);
                    Trow[0] = make_float2(2.0f * fs.x, 2.0f * fs.y);  // 2s
                    Trow[1] = make_float2(1.0f, 0.0f);                // T_0
                    Trow[1 + nq] = fs;                                // T_1
                    if (A.stab) {
                        // T_4i and T_4i+1 (the direct path stored them above) by the
                        // recurrence of stride 4, X_(i+1) = 2 T_4 X_i - X_(i-1) (from
                        // T_(m+4) + T_(m-4) = 2 T_4 T_m), in double-float from T_4 and T_5
                        // formed in FP64: the rounding errors (2^-48 per step) grow at most
                        // like i^2 over i steps, below 2 i^2 2^-48 for |s| <= 1
                        const double T2 = fma(2.0 * s, s, -1.0);
                        const double T3 = fma(2.0 * s, T2, -s);
                        const double T4 = fma(2.0 * T2, T2, -1.0);
                        const float2 c4 = df_split(2.0 * T4, 0);
                        float2 a0 = make_float2(1.0f, 0.0f), a1 = df_split(T4, 0);  // T_(4i-4), T_4i
                        float2 b0 = fs, b1 = df_split(fma(2.0 * s, T4, -T3), 0);    // T_(4i-3), T_(4i+1)
                        for (int i = 1; i < nq; ++i) {
                            Trow[1 + i] = a1;
                            Trow[1 + nq + i] = b1;
                            const float2 an4 = df_mulsub(c4, a1, a0);
                            a0 = a1;
                            a1 = an4;
                            const float2 bn = df_mulsub(c4, b1, b0);
                            b0 = b1;
                            b1 = bn;
                        }
                    }
                }
                const double Kw = f[2] * (an.w * an.s4);
                if (ghost) hG = Kw * Zz * iz2;
                if (gluon) {
                    const double sg = an.sig;
                    const double num = fma(sg, fma(sg, fma(sg, fma(sg, f[7], f[6]), f[5]), f[4]), f[3]);
                    hQ = (an.w * an.s2) * iz2 * Wz * num;
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
                        const float2 s2 = AR ? Tm[0] : make_float2(0.0f, 0.0f);
#pragma unroll
                        for (int jj = 0; jj < NJ; ++jj) {
                            if (colj[jj] < N) {
                                float2 t;
                                if (AR) {
                                    const float2 a = Tm[1 + coli[jj]];
                                    const float2 b = Tm[1 + nq + coli[jj]];
                                    t = (colr[jj] & 1) ? b : a;
                                    if (colr[jj] >= 2) {
                                        const float2 t2 = df_mulsub(s2, b, a);
                                        t = colr[jj] == 2 ? t2 : df_mulsub(s2, t2, b);
                                    }
                                    if (colj[jj] == 0) t = make_float2(0.5f, 0.0f);  // T_0 enters as 1/2
                                } else {
                                    t = Tm[colj[jj]];
                                }
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

template <int BT, int NJ, bool FULL>
__global__ void __launch_bounds__(BT) k_triple(const __grid_constant__ TripleArgs A) {
    extern __shared__ __align__(16) double smem[];
    triple_tile<BT, NJ, FULL, kAnchorRowsSingle>(A, blockIdx.y, blockIdx.x, smem);
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
        triple_tile<BT, NJ, FULL, kAnchorRowsBatched>(A, w.rt, w.ks, smem);
    }
}

template <int BT, bool FULL>
cudaError_t launch_bt(const TripleArgs& a, cudaStream_t s) {
    const int N = a.c.N;
    const size_t smem = smem_doubles(FULL, N, BT, kAnchorRowsSingle) * sizeof(double);
    const dim3 grid(a.KS, a.Rt);
    const int nj = (N + BT - 1) / BT;
    cudaError_t e = cudaSuccess;
    if (nj <= 1) {
        e = cudaFuncSetAttribute(k_triple<BT, 1, FULL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_triple<BT, 1, FULL><<<grid, BT, smem, s>>>(a);
    } else if (nj <= 2) {
        e = cudaFuncSetAttribute(k_triple<BT, 2, FULL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_triple<BT, 2, FULL><<<grid, BT, smem, s>>>(a);
    } else if (nj <= 4) {
        e = cudaFuncSetAttribute(k_triple<BT, 4, FULL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_triple<BT, 4, FULL><<<grid, BT, smem, s>>>(a);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int BT, bool FULL>
int occupancy_bt(int N) {
    const size_t smem = smem_doubles(FULL, N, BT, kAnchorRowsSingle) * sizeof(double);
    const int nj = (N + BT - 1) / BT;
    int nb = 0;
    cudaError_t e;
    if (nj <= 1) {
        cudaFuncSetAttribute(k_triple<BT, 1, FULL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_triple<BT, 1, FULL>, BT, smem);
    } else if (nj <= 2) {
        cudaFuncSetAttribute(k_triple<BT, 2, FULL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_triple<BT, 2, FULL>, BT, smem);
    } else {
        cudaFuncSetAttribute(k_triple<BT, 4, FULL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_triple<BT, 4, FULL>, BT, smem);
    }
    return e == cudaSuccess ? nb : 0;
}

}  // namespace

int triple_block_threads(int N) { return block_threads_for(N); }

size_t triple_smem_bytes(bool full, int N) {
    return smem_doubles(full, N, block_threads_for(N), kAnchorRowsSingle) * sizeof(double);
}

int triple_max_blocks_per_sm(bool full, int N) {
    if (block_threads_for(N) == 128) return full ? occupancy_bt<128, true>(N) : occupancy_bt<128, false>(N);
    return full ? occupancy_bt<64, true>(N) : occupancy_bt<64, false>(N);
}

namespace {
template <int BT, bool FULL>
cudaError_t launch_batched_bt(const BatchProblem* P, const BatchItem* items, int n_items, int* counter,
                              const double* coef_base, int maxN, int grid, cudaStream_t s) {
    const size_t smem = smem_doubles(FULL, maxN, BT, kAnchorRowsBatched) * sizeof(double);
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
    const size_t smem = smem_doubles(FULL, maxN, BT, kAnchorRowsBatched) * sizeof(double);
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
    if (block_threads_for(a.c.N) == 128) return full ? launch_bt<128, true>(a, s) : launch_bt<128, false>(a, s);
    return full ? launch_bt<64, true>(a, s) : launch_bt<64, false>(a, s);
}

}  // namespace dse
