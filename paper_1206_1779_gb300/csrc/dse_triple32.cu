// dse_triple32.cu -- the quadrature kernel of the mixed-precision Newton matrix
// (precision = 1).
//
// Same outputs and layouts as the FP64 kernel of dse_triple.cu (Upart, Vpart in
// FP64), with the precision split of the mixed-precision Newton matrix:
//   FP64: the Chebyshev log-momentum map s(z) = (ln z - L0)/L1 (z, ln z and the
//         distance 1 - |s| to the ends of the interval, which the FP32 recurrence
//         for T_j needs to full relative accuracy); the exponentials of the
//         dressing-function series, taken at the nodes of the series table (the
//         kernel interpolates Z, G and W = G^p Z^q from it) and, for z outside
//         [eps2, lambda2], per triple; the angular and radial sums beyond one
//         block of triples (Upart, Vpart, and their FP64 contraction after it).
//   FP32: 1/z, the table polynomials, the kernels M and Q and the three
//         integrands, T_j(s) by the forward recurrence in differences,
//           D_(j+1) = sgn(s) (D_j - 2 (1 - |s|) T_j),  T_(j+1) = sgn(s) T_j + D_(j+1),
//         whose rounding errors grow like j rather than j^2 near s = +-1, and the
//         products weight * T_j;
//   compensated (two-sum) block accumulation: each thread adds its products over
//   blocks of 8 triples in FP32 and joins each block sum to a compensated pair
//   (sum, error) by Knuth's two-sum, which is widened to FP64 at the end.
// The Jacobian built from these sums carries relative errors of about 1e-7 of the
// entries' magnitude sums; the mixed-precision Newton iteration pairs it with an
// FP64 residual near convergence (an inexact Newton method whose fixed point is
// the FP64 solution).
//
// Tile layout: one block of BT threads per (row, radial split) walks its radial
// nodes in tiles of BT triples (one warp = 32 angular nodes of one radial node).
// Shared-memory row of triple m (float4 units, stride rs4 = quad count + 1 made
// odd): [0] (hQ, hM, hG, 0), [1 + i] (T_4i .. T_4i+3) with T_0 stored as 1/2.
// Thread (group g, quad i) then sums the twelve products of its four columns over
// the rows of group g.
#include "dse_internal.cuh"
#include "dse_lnrcp.cuh"

namespace dse {

namespace {

constexpr unsigned kFullMask32 = 0xffffffffu;
constexpr double kPi32 = 3.14159265358979323846264338327950288;

__host__ __device__ inline int bt32_for(int N) { return N <= 128 ? 128 : 64; }
__host__ __device__ inline int quads32(int N) { return (N + 3) / 4; }
__host__ __device__ inline int stride32(int N) { return (quads32(N) + 1) | 1; }

// radial-node factors: d, 4 sqrt(xy) (FP64, for z), K = W_k y G(y) and the five
// quartic coefficients of the gluon-loop kernel times W_k W(y)/2 (FP32)
constexpr int kRadGroup32 = 32;
struct RadF32 { double d, b2; float K, q0, q1, q2, q3, q4, pad0, pad1; };

__host__ __device__ inline size_t smem32_bytes(int N, int BT, int KB) {
    const int kg = KB < kRadGroup32 ? KB : kRadGroup32;
    const size_t tile = (size_t)BT * stride32(N) * sizeof(float4);
    const size_t red = (size_t)(BT / quads32(N)) * 3u * (size_t)N * sizeof(double2);
    return (tile > red ? tile : red) + 2u * (size_t)N * sizeof(float) + 4u * sizeof(double) +
           (size_t)kg * sizeof(RadF32);
}

// 2^d as FP32 (0 below the normal range, Inf above it)
__device__ __forceinline__ float pow2f32(int d) {
    return d < -126 ? 0.0f : d > 127 ? __int_as_float(0x7f800000) : __int_as_float((127 + d) << 23);
}

// c += t in the compensated pair (c.x the sum, c.y the accumulated rounding errors)
__device__ __forceinline__ void two_sum_acc(float2& c, const float t) {
    const float s = c.x + t;
    const float bb = s - c.x;
    c.y += (c.x - (s - bb)) + (t - bb);
    c.x = s;
}

template <int BT>
__global__ void __launch_bounds__(BT) k_triple32(const __grid_constant__ TripleArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Consts& c = A.c;
    const int N = c.N;
    const int nq = quads32(N);
    const int rs4 = stride32(N);
    constexpr int WARPS = BT / 32;
    float4* sT = reinterpret_cast<float4*>(smem_raw);
    const size_t tile_bytes = (size_t)BT * rs4 * sizeof(float4);
    const size_t red_bytes = (size_t)(BT / nq) * 3u * (size_t)N * sizeof(double2);
    float* sa = reinterpret_cast<float*>(smem_raw + (tile_bytes > red_bytes ? tile_bytes : red_bytes));
    float* sb = sa + N;
    double* sbnd = reinterpret_cast<double*>(sb + N);  // (2 N floats: 8-byte aligned)
    RadF32* srad = reinterpret_cast<RadF32*>(sbnd + 4);
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;

    // the series' coefficients (for N below the table's range), zero-padded to N
    for (int j = tid; j < N; j += BT) {
        sa[j] = j < c.NZ ? (float)A.coef[j] : 0.0f;
        sb[j] = j < c.NG ? (float)A.coef[c.NZ + j] : 0.0f;
    }
    if (A.stab && tid < 4) sbnd[tid] = reinterpret_cast<const double*>(A.stab + kSeriesM)[tid];
    const int rt = blockIdx.y;
    const int ks = blockIdx.x;
    const Row row = A.rows[rt];
    const bool gluon = (row.flags & kRowGluon) != 0;
    const bool ghost = (row.flags & kRowGhost) != 0;
    const int k0 = ks * A.KB;
    const int k1 = min(c.nr, k0 + A.KB);
    const int nch = A.nch;
    const int nunits = k1 > k0 ? (k1 - k0) * nch : 0;
    const int kgrp = A.KB < kRadGroup32 ? A.KB : kRadGroup32;
    const float ith_scale = (float)c.sM * (float)(1.0 / kPi32);

    // phase-B mapping: G groups of nq threads, rows [g R, (g + 1) R)
    const int G = BT / nq;
    const int R = (BT + G - 1) / G;
    const int g = tid / nq;
    const int qi = tid - g * nq;
    const bool bact = g < G;
    const int mlo = min(BT, g * R);
    const int mhi = min(BT, mlo + R);
    float2 acc[3][4];  // compensated pairs (sum, error)
#pragma unroll
    for (int kd = 0; kd < 3; ++kd)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[kd][q] = make_float2(0.0f, 0.0f);

    const int group_units = kgrp * nch;
    for (int base = 0; base < nunits; base += WARPS) {
        if (base % group_units == 0) {
            __syncthreads();  // the previous group's factors are no longer read (and the coefficients staged)
            const int kq = k0 + base / nch + lane;
            if (warp == 0 && lane < kgrp && kq < k1) {
                const Rad rd = A.rad[rad_offset(c, rt) + kq];
                const YTab yt = A.ytab[rad_offset(c, rt) + kq];
                const double d0 = row.sx - rd.sy;
                const double d = d0 * d0;
                const double b = 2.0 * row.sx * rd.sy;
                const double dd = d * d, db = d * b, bb = b * b;
                const double h = 0.5 * rd.W * yt.Wy;
                RadF32 f;
                f.d = d;
                f.b2 = 2.0 * b;
                f.K = (float)(rd.W * yt.yG);
                f.q0 = (float)(h * (7.5 * dd));
                f.q1 = (float)(h * -(48.0 * dd + 18.0 * db + 12.0 * bb));
                f.q2 = (float)(h * (48.0 * dd - 48.0 * db - 38.0 * bb));
                f.q3 = (float)(h * (96.0 * db + 64.0 * bb));
                f.q4 = (float)(h * (16.0 * bb));
                f.pad0 = f.pad1 = 0.0f;
                srad[lane] = f;
            }
            __syncthreads();
        }
        const int u = base + warp;
        float hQ = 0.0f, hM = 0.0f, hG = 0.0f;
        float4* Trow = sT + (size_t)tid * rs4;
        bool live = false;
        int k = 0, ch = 0;
        if (u < nunits) {
            const int kk = u / nch;
            ch = u - kk * nch;
            k = k0 + kk;
            const int l = ch * 32 + lane;
            if (l < c.na) {
                live = true;
                const RadF32& f = srad[kk % kgrp];
                const Ang an = A.ang[l];
                // the map in FP64: z, ln z, s and 1 - |s|
                const double z = fma(f.b2, an.sig, f.d);
                const LnRcp lr = ln_rcp(z);
                double sd = (lr.ln - c.L0) * c.invL1;
                const long long zb = __double_as_longlong(z);
                const bool beyond = zb < __double_as_longlong(c.eps2) || zb > __double_as_longlong(c.lam2);
                const bool outside = c.extrap == 0 && beyond;
                if (beyond) sd = fmin(1.0, fmax(-1.0, sd));
                const float s = (float)sd;
                const float m2d = (float)(-2.0 * (1.0 - fabs(sd)));  // -2 (1 - |s|), relative accuracy
                const float sg = sd < 0.0 ? -1.0f : 1.0f;
                // T_j(s) by the recurrence in differences, written to the row as quads
                // (T_0 as 1/2); for N below the table's range the series as well
                const bool series = A.stab == nullptr;
                float lg = 0.0f, lzz = 0.0f;
                if (series) {
                    lg = 0.5f * sb[0];
                    lzz = 0.5f * sa[0];
                    if (N > 1) {
                        lg = fmaf(sb[1], s, lg);
                        lzz = fmaf(sa[1], s, lzz);
                    }
                }
                {
                    float T = s;        // T_1
                    float D = s - sg;   // D_1 = T_1 - sgn(s) T_0
                    float4 qv = make_float4(0.5f, s, 0.0f, 0.0f);
                    for (int j = 2; j < 4 * nq; ++j) {
                        D = sg * fmaf(m2d, T, D);
                        T = fmaf(sg, T, D);
                        if (series && j < N) {
                            lg = fmaf(sb[j], T, lg);
                            lzz = fmaf(sa[j], T, lzz);
                        }
                        const float tv = j < N ? T : 0.0f;
                        if ((j & 3) == 2) qv.z = tv;
                        else if ((j & 3) == 3) {
                            qv.w = tv;
                            Trow[1 + (j >> 2)] = qv;
                        } else if ((j & 3) == 0) qv.x = tv;
                        else qv.y = tv;
                    }
                }
                // the dressing functions at z
                float Zz = 0.0f, Gz = 0.0f, Wz = 0.0f;
                if (A.stab && !outside) {
                    // from the series table, built from FP64 exponentials at its nodes:
                    // the polynomials' leading parts in FP32, scaled by the records'
                    // exponents
                    const float sf = fminf(1.0f, fmaxf(-1.0f, s));
                    int it = (int)(acosf(sf) * ith_scale);
                    it = min(max(it, 0), c.sM - 1);
                    const SeriesRec* Rr = A.stab + it;
                    const double2 mh = __ldg(reinterpret_cast<const double2*>(Rr));
                    const float uu = (float)((sd - mh.x) * mh.y);
                    const int4 ex = __ldg(reinterpret_cast<const int4*>(Rr->ex));
                    if (ghost || gluon) {
                        const float4 top = __ldg(&Rr->e[kSeriesP]);
                        float tz = top.x, tg = top.y;
#pragma unroll
                        for (int q = kSeriesP - 1; q >= 0; --q) {
                            const float4 ck = __ldg(&Rr->e[q]);
                            tz = fmaf(tz, uu, ck.x);
                            tg = fmaf(tg, uu, ck.y);
                        }
                        Zz = tz * pow2f32(ex.x - 1023);
                        Gz = tg * pow2f32(ex.y - 1023);
                    }
                    if (gluon) {
                        float tw = __ldg(&Rr->w[kSeriesP]).x;
#pragma unroll
                        for (int q = kSeriesP - 1; q >= 0; --q) tw = fmaf(tw, uu, __ldg(&Rr->w[q]).x);
                        Wz = tw * pow2f32(ex.z - 1023);
                    }
                } else {
                    // outside [eps2, lambda2] (or no table): the series' values in FP64,
                    // the IR/UV forms and the exponentials in FP64
                    double lgd, lzd;
                    if (A.stab) {
                        lzd = sd > 0.0 ? sbnd[0] : sbnd[2];
                        lgd = sd > 0.0 ? sbnd[1] : sbnd[3];
                    } else {
                        lgd = lg;
                        lzd = lzz;
                    }
                    if (outside) {
                        if (z < c.eps2) {
                            const double r = lr.ln - c.ln_eps2;
                            lgd = fma(-c.kappa, r, lgd);
                            lzd = fma(2.0 * c.kappa, r, lzd);
                        } else {
                            const double L = log1p(c.omega * (lr.ln - c.ln_lam2));
                            lgd = fma(c.delta, L, lgd);
                            lzd = fma(c.gam, L, lzd);
                        }
                    }
                    if (ghost) Zz = (float)exp(lzd);
                    if (gluon) {
                        Gz = (float)exp(lgd);
                        Wz = (float)exp(c.pG * lgd + c.qZ * lzd);
                    }
                }
                // the integrands in FP32
                const float zf = (float)z;
                const float iz = 1.0f / zf;
                const float iz2 = iz * iz;
                const float Kw = f.K * (float)an.ws4;
                if (ghost) hG = (Kw * iz2) * Zz;
                if (gluon) {
                    const float sgm = (float)an.sig;
                    const float num = fmaf(sgm, fmaf(sgm, fmaf(sgm, fmaf(sgm, f.q4, f.q3), f.q2), f.q1), f.q0);
                    hQ = ((float)an.ws2 * iz2) * Wz * num;
                    hM = (Kw * iz) * Gz;
                }
            }
        }
        if (!live) {
            for (int i = 1; i <= nq; ++i) Trow[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
        Trow[0] = make_float4(hQ, hM, hG, 0.0f);
        // angular sums over the warp's 32 nodes (FP32; the radial sums beyond are FP64)
        {
            float rQ = hQ, rM = hM, rG = hG;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                rQ += __shfl_xor_sync(kFullMask32, rQ, off);
                rM += __shfl_xor_sync(kFullMask32, rM, off);
                rG += __shfl_xor_sync(kFullMask32, rG, off);
            }
            if (u < nunits && lane == 0) {
                double* up = A.Upart + (((size_t)rt * c.nr + k) * nch + ch) * 3;
                up[0] = (double)rQ;
                up[1] = (double)rM;
                up[2] = (double)rG;
            }
        }
        __syncthreads();
        if (bact) {
            // blocks of 8 rows summed in FP32, each block joined to the compensated pairs
            for (int m0 = mlo; m0 < mhi; m0 += 8) {
                const int m1 = min(mhi, m0 + 8);
                float p[3][4];
#pragma unroll
                for (int kd = 0; kd < 3; ++kd)
#pragma unroll
                    for (int q = 0; q < 4; ++q) p[kd][q] = 0.0f;
                for (int m = m0; m < m1; ++m) {
                    const float4* Tm = sT + (size_t)m * rs4;
                    const float4 h = Tm[0];
                    const float4 t = Tm[1 + qi];
                    p[0][0] = fmaf(h.x, t.x, p[0][0]);
                    p[0][1] = fmaf(h.x, t.y, p[0][1]);
                    p[0][2] = fmaf(h.x, t.z, p[0][2]);
                    p[0][3] = fmaf(h.x, t.w, p[0][3]);
                    p[1][0] = fmaf(h.y, t.x, p[1][0]);
                    p[1][1] = fmaf(h.y, t.y, p[1][1]);
                    p[1][2] = fmaf(h.y, t.z, p[1][2]);
                    p[1][3] = fmaf(h.y, t.w, p[1][3]);
                    p[2][0] = fmaf(h.z, t.x, p[2][0]);
                    p[2][1] = fmaf(h.z, t.y, p[2][1]);
                    p[2][2] = fmaf(h.z, t.z, p[2][2]);
                    p[2][3] = fmaf(h.z, t.w, p[2][3]);
                }
#pragma unroll
                for (int kd = 0; kd < 3; ++kd)
#pragma unroll
                    for (int q = 0; q < 4; ++q) two_sum_acc(acc[kd][q], p[kd][q]);
            }
        }
        __syncthreads();
    }

    // combine the groups in FP64 in a fixed order and write this block's split
    double2* red = reinterpret_cast<double2*>(smem_raw);  // [G][3][N]: (sum, error) widened
    if (bact) {
#pragma unroll
        for (int kd = 0; kd < 3; ++kd)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = 4 * qi + q;
                if (j < N) red[((size_t)g * 3 + kd) * N + j] = make_double2(acc[kd][q].x, acc[kd][q].y);
            }
    }
    __syncthreads();
    double* out = A.Vpart + ((size_t)rt * A.KS + ks) * 3 * (size_t)N;
    for (int idx = tid; idx < 3 * N; idx += BT) {
        double v = 0.0;
        for (int gg = 0; gg < G; ++gg) {
            const double2 r = red[(size_t)gg * 3 * N + idx];
            v += r.x + r.y;
        }
        out[idx] = v;
    }
}

template <int BT>
cudaError_t launch32_bt(const TripleArgs& a, cudaStream_t s) {
    const size_t smem = smem32_bytes(a.c.N, BT, a.KB);
    const dim3 grid(a.KS, a.Rt);
    cudaError_t e = cudaFuncSetAttribute(k_triple32<BT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_triple32<BT><<<grid, BT, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

// Newton-matrix mode only (the mixed-precision residual is the FP64 kernel's).
cudaError_t launch_triple32(bool full, const TripleArgs& a, cudaStream_t s) {
    if (!full) return cudaErrorInvalidValue;
    if (a.KS <= 0 || a.Rt <= 0) return cudaSuccess;
    return bt32_for(a.c.N) == 128 ? launch32_bt<128>(a, s) : launch32_bt<64>(a, s);
}

}  // namespace dse
