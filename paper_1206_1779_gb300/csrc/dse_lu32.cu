// dse_lu32.cu -- the Newton step (Sec. 3: J Delta = F, c <- c - rho Delta) for
// n = N_Z + N_G above the register Gauss-Jordan's range (160 < n <= 2 DSE_MAX_CHEB):
// an FP32 LU factorisation with partial pivoting of the row-scaled matrix
// A = diag(s) J (k_scale_rows: s_i the power of two that brings row i's largest
// entry into [1/2, 1)), then FP64 iterative refinement x <- x + U^-1 L^-1 P s (F - J x)
// with the residual in FP64, until max |s (F - J x)| <= 4 sqrt(n) 2^-53 ||A|| max|x|
// (a backward-stable solution).  One block of 1024 threads; the FP64 LU of
// k_lu_newton takes over when a pivot is zero or the refinement stops contracting.
//
// The factorisation is blocked (panels of kPB columns, right-looking):
//   - a panel (all rows at and below it) is factored in shared memory, column by
//     column: the pivot is the largest magnitude of the column (one block-wide
//     max over 32-bit keys: the magnitude's bits above 9 and 511 - row, so that
//     of magnitudes within 2^-14 of each other the lowest row wins);
//   - rows are never moved in memory: the row order lives in perm (logical row ->
//     physical row of As), and a pivot swaps two entries of perm and two rows of
//     the panel in shared memory;
//   - U12 = L11^-1 A12 by one thread per column, then A22 -= L21 U12 from shared
//     memory, 4 x 4 entries per thread.
// The triangular solves of a sweep go by blocks of 32 rows: one warp solves the
// diagonal block by shuffles, then every thread updates the rows below (above).
#include "dse_internal.cuh"

namespace dse {

namespace {

constexpr unsigned kFM = 0xffffffffu;
constexpr int kLuT = 1024;         // threads
constexpr int kPB = 32;            // panel width
constexpr int kLuSweeps = 12;      // refinement sweeps at most
constexpr double kLuRate = 0.5;    // a sweep must reduce the residual by this factor
constexpr int kLuMaxN = 2 * DSE_MAX_CHEB;

__host__ __device__ inline int lu_ld(int n) { return ((n + 3) & ~3) + 4; }  // panel / U12 row stride

__global__ void __launch_bounds__(kLuT) k_newton_lu32(const Consts c, const double* __restrict__ J,
                                                      float* __restrict__ As, const double2* __restrict__ rowinfo,
                                                      const double* __restrict__ F, const XTab* __restrict__ xtab,
                                                      double* __restrict__ coef, const double rho,
                                                      double* __restrict__ stats, int* __restrict__ status,
                                                      int* __restrict__ done) {
    extern __shared__ __align__(16) double lsm[];
    const int n = c.n;
    const int ld = lu_ld(n);
    float* Pc = reinterpret_cast<float*>(lsm);          // [kPB][ld] panel, column-major (16-byte rows)
    float* Uc = Pc + (size_t)kPB * ld;                  // [kPB][ld] U12 rows
    float* zf = Uc + (size_t)kPB * ld;                  // [ld] FP32 right-hand side / solution
    double* xs = reinterpret_cast<double*>(zf + ld);    // [n] solution (ld is a multiple of 4)
    double* rs = xs + n;                                // [n] FP64 residual
    double* Ss = rs + n;                                // [n] row scales
    int* perm = reinterpret_cast<int*>(Ss + n);         // [n] logical -> physical row
    __shared__ unsigned s_key[kLuT / 32];
    __shared__ double s_red[2][kLuT / 32];
    __shared__ unsigned s_pk;
    __shared__ int s_fail, s_conv, s_ok;
    __shared__ double s_anorm, s_prev;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int WARPS = kLuT / 32;

    // norms of F, ||A||_inf, row scales, identity order
    if (warp == 0) {
        double mF = 0.0, mS = 0.0, an = 0.0;
        bool bad = false;
        for (int i = lane; i < n; i += 32) {
            const double f = F[i];
            const double sc = i < c.NZ ? xtab[i].Z : xtab[c.gofs + i - c.NZ].G;
            mF = fmax(mF, fabs(f));
            mS = fmax(mS, fabs(f) * sc);
            bad |= !isfinite(f);
            an = fmax(an, rowinfo[i].y);
        }
        for (int off = 16; off > 0; off >>= 1) {
            mF = fmax(mF, __shfl_xor_sync(kFM, mF, off));
            mS = fmax(mS, __shfl_xor_sync(kFM, mS, off));
            an = fmax(an, __shfl_xor_sync(kFM, an, off));
        }
        bad = __any_sync(kFM, bad);
        if (lane == 0) {
            stats[0] = bad ? INFINITY : mF;
            stats[1] = mS;
            stats[2] = 0.0;
            stats[3] = -1.0;
            s_anorm = an;
            s_fail = ((*status) & (kStatusNonfinite | kStatusSingular)) | (bad ? kStatusNonfinite : 0);
            s_prev = INFINITY;
        }
    }
    for (int i = tid; i < n; i += kLuT) {
        Ss[i] = rowinfo[i].x;
        perm[i] = i;
        xs[i] = 0.0;
        rs[i] = F[i];
    }
    __syncthreads();
    if (s_fail) {
        // non-finite F or a flagged J: reported as they are, no fallback
        if (tid == 0) {
            atomicOr(status, s_fail);
            *done = 1;
        }
        return;
    }

    // ---------------- FP32 LU with partial pivoting ----------------
    bool lu_ok = true;
    for (int p = 0; p < n && lu_ok; p += kPB) {
        const int w = min(kPB, n - p);
        const int m = n - p;
        for (int idx = tid; idx < m * kPB; idx += kLuT) {
            const int i = idx >> 5, cc = idx & 31;
            if (cc < w) Pc[cc * ld + i] = As[(size_t)perm[p + i] * n + p + cc];
        }
        __syncthreads();
        for (int k = 0; k < w; ++k) {
            unsigned key = 0u;
            for (int i = k + tid; i < m; i += kLuT) {
                const unsigned b = __float_as_uint(fabsf(Pc[k * ld + i]));
                key = max(key, (b & 0xfffffe00u) | (unsigned)(511 - i));
            }
            key = __reduce_max_sync(kFM, key);
            if (lane == 0) s_key[warp] = key;
            __syncthreads();
            if (warp == 0) {
                unsigned kk = s_key[lane];
                kk = __reduce_max_sync(kFM, kk);
                if (lane == 0) {
                    const int ip0 = 511 - (int)(kk & 511u);
                    const float pv = Pc[k * ld + ip0];
                    s_pk = (unsigned)ip0;
                    s_ok = (fabsf(pv) > 0.0f && isfinite(pv)) ? 1 : 0;
                }
            }
            __syncthreads();
            if (!s_ok) {
                lu_ok = false;  // uniform: one thread decided, every thread reads the decision
                break;
            }
            const int ip = (int)s_pk;
            if (ip != k) {
                if (tid < w) {
                    const float t = Pc[tid * ld + k];
                    Pc[tid * ld + k] = Pc[tid * ld + ip];
                    Pc[tid * ld + ip] = t;
                }
                if (tid == 0) {
                    const int t = perm[p + k];
                    perm[p + k] = perm[p + ip];
                    perm[p + ip] = t;
                }
            }
            __syncthreads();
            const float rd = 1.0f / Pc[k * ld + k];
            for (int i = k + 1 + tid; i < m; i += kLuT) {
                const float l = Pc[k * ld + i] * rd;
                Pc[k * ld + i] = l;
                for (int cc = k + 1; cc < w; ++cc) Pc[cc * ld + i] = fmaf(-l, Pc[cc * ld + k], Pc[cc * ld + i]);
            }
            __syncthreads();
        }
        if (!lu_ok) break;
        // the factored panel back to its rows (physical rows are never moved)
        for (int idx = tid; idx < m * kPB; idx += kLuT) {
            const int i = idx >> 5, cc = idx & 31;
            if (cc < w) As[(size_t)perm[p + i] * n + p + cc] = Pc[cc * ld + i];
        }
        const int m2 = n - p - w;  // trailing size
        if (m2 > 0) {
            // U12 = L11^-1 A12, one thread per column
            for (int jc = tid; jc < m2; jc += kLuT) {
                const int j = p + w + jc;
                float u[kPB];
#pragma unroll
                for (int kk = 0; kk < kPB; ++kk) u[kk] = kk < w ? As[(size_t)perm[p + kk] * n + j] : 0.0f;
#pragma unroll
                for (int kk = 1; kk < kPB; ++kk) {
#pragma unroll
                    for (int l = 0; l < kk; ++l) u[kk] = fmaf(-Pc[l * ld + kk], u[l], u[kk]);
                }
#pragma unroll
                for (int kk = 0; kk < kPB; ++kk) {
                    if (kk < w) As[(size_t)perm[p + kk] * n + j] = u[kk];
                    Uc[kk * ld + jc] = u[kk];
                }
            }
            __syncthreads();
            // A22 -= L21 U12 (w = kPB here: the trailing part exists only below a full panel)
            const int nt = (m2 + 3) >> 2;
            for (int t = tid; t < nt * nt; t += kLuT) {
                const int r0 = (t / nt) * 4, c0 = (t % nt) * 4;
                float acc[4][4];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
#pragma unroll 4
                for (int kk = 0; kk < kPB; ++kk) {
                    const float4 la = *reinterpret_cast<const float4*>(&Pc[kk * ld + w + r0]);
                    const float4 ub = *reinterpret_cast<const float4*>(&Uc[kk * ld + c0]);
                    const float lv[4] = {la.x, la.y, la.z, la.w};
                    const float uv[4] = {ub.x, ub.y, ub.z, ub.w};
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(lv[a], uv[b], acc[a][b]);
                }
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    if (r0 + a >= m2) break;
                    float* row = As + (size_t)perm[p + w + r0 + a] * n + p + w;
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        if (c0 + b < m2) row[c0 + b] -= acc[a][b];
                }
            }
        }
        __syncthreads();
    }

    // ---------------- FP64 iterative refinement ----------------
    int sweeps = 0;
    int verdict = lu_ok ? 0 : 2;  // 0 running, 1 converged, 2 gave up
    const double tolfac = 4.0 * sqrt((double)n) * 0x1p-53 * s_anorm;
    while (verdict == 0) {
        // right-hand side in the logical order: s r
        for (int i = tid; i < n; i += kLuT) {
            const int pr = perm[i];
            zf[i] = (float)(Ss[pr] * rs[pr]);
        }
        __syncthreads();
        // forward: L z = P s r (unit lower), blocks of 32 rows
        for (int q = 0; q < n; q += 32) {
            const int bw = min(32, n - q);
            if (warp == 0) {
                float lrow[32];
                const int pr = lane < bw ? perm[q + lane] : 0;
#pragma unroll
                for (int cc = 0; cc < 32; ++cc) lrow[cc] = (lane < bw && cc < lane) ? As[(size_t)pr * n + q + cc] : 0.0f;
                float z = lane < bw ? zf[q + lane] : 0.0f;
#pragma unroll
                for (int cc = 0; cc < 32; ++cc) {
                    const float zc = __shfl_sync(kFM, z, cc);
                    if (cc < lane) z = fmaf(-lrow[cc], zc, z);
                }
                if (lane < bw) zf[q + lane] = z;
            }
            __syncthreads();
            for (int i = q + bw + tid; i < n; i += kLuT) {
                const float* Lr = As + (size_t)perm[i] * n + q;
                float s = zf[i];
                for (int cc = 0; cc < bw; ++cc) s = fmaf(-Lr[cc], zf[q + cc], s);
                zf[i] = s;
            }
            __syncthreads();
        }
        // backward: U dx = z, blocks of 32 rows from the bottom
        for (int q = ((n - 1) / 32) * 32; q >= 0; q -= 32) {
            const int bw = min(32, n - q);
            if (warp == 0) {
                float urow[32];
                const int pr = lane < bw ? perm[q + lane] : 0;
#pragma unroll
                for (int cc = 0; cc < 32; ++cc) urow[cc] = (lane < bw && cc >= lane && cc < bw) ? As[(size_t)pr * n + q + cc] : 0.0f;
                float z = lane < bw ? zf[q + lane] : 0.0f;
#pragma unroll
                for (int cc = 31; cc >= 0; --cc) {
                    if (cc < bw && lane == cc) z = z / urow[cc];
                    const float zc = __shfl_sync(kFM, z, cc);
                    if (cc < bw && lane < cc) z = fmaf(-urow[cc], zc, z);
                }
                if (lane < bw) zf[q + lane] = z;
            }
            __syncthreads();
            for (int i = tid; i < q; i += kLuT) {
                const float* Ur = As + (size_t)perm[i] * n + q;
                float s = zf[i];
                for (int cc = 0; cc < bw; ++cc) s = fmaf(-Ur[cc], zf[q + cc], s);
                zf[i] = s;
            }
            __syncthreads();
        }
        for (int i = tid; i < n; i += kLuT) xs[i] += (double)zf[i];
        ++sweeps;
        __syncthreads();
        // FP64 residual r = F - J x: two threads per row (n <= 512 rows)
        double rm = 0.0, xm = 0.0;
        {
            const int row = tid >> 1, hf = tid & 1;
            double acc = 0.0;
            if (row < n) {
                const double* Jr = J + (size_t)row * n;
                const int j0 = hf ? n / 2 : 0, j1 = hf ? n : n / 2;
                double a0 = 0.0, a1 = 0.0;
                int jj = j0;
                for (; jj + 1 < j1; jj += 2) {
                    a0 = fma(Jr[jj], xs[jj], a0);
                    a1 = fma(Jr[jj + 1], xs[jj + 1], a1);
                }
                if (jj < j1) a0 = fma(Jr[jj], xs[jj], a0);
                acc = a0 + a1;
            }
            acc += __shfl_xor_sync(kFM, acc, 1);
            if (row < n && hf == 0) {
                const double r = F[row] - acc;
                rs[row] = r;
                const double rn = Ss[row] * r;
                rm = isfinite(rn) ? fabs(rn) : INFINITY;
                xm = fabs(xs[row]);
            }
        }
        for (int off = 16; off > 0; off >>= 1) {
            rm = fmax(rm, __shfl_xor_sync(kFM, rm, off));
            xm = fmax(xm, __shfl_xor_sync(kFM, xm, off));
        }
        if (lane == 0) {
            s_red[0][warp] = rm;
            s_red[1][warp] = xm;
        }
        __syncthreads();
        if (tid == 0) {
            double RM = 0.0, XM = 0.0;
            for (int w = 0; w < WARPS; ++w) {
                RM = fmax(RM, s_red[0][w]);
                XM = fmax(XM, s_red[1][w]);
            }
            int v = 0;
            if (!isfinite(RM) || !isfinite(XM)) v = 2;
            else if (RM <= tolfac * XM) v = 1;
            else if (sweeps >= kLuSweeps || !(RM <= kLuRate * s_prev)) v = 2;
            s_prev = RM;
            s_conv = v;
            if (v == 1) stats[2] = XM;
        }
        __syncthreads();
        verdict = s_conv;
    }
    if (verdict != 1) {
        // the FP64 LU of k_lu_newton takes the step (J and F are untouched)
        if (tid == 0) *done = 0;
        return;
    }
    for (int i = tid; i < n; i += kLuT) coef[i] = fma(-rho, xs[i], coef[i]);
    if (tid == 0) {
        stats[3] = (double)sweeps;
        *done = 1;
    }
}

}  // namespace

size_t newton_lu32_smem_bytes(int n) {
    const int ld = lu_ld(n);
    return sizeof(double) * 3 * (size_t)n + sizeof(float) * (2 * (size_t)kPB * ld + ld) + sizeof(int) * (size_t)n;
}

cudaError_t launch_newton_lu32(const Consts& c, const double* J, float* As, const double2* rowinfo, const double* F,
                               const XTab* xtab, double* coef, double rho, double* stats, int* status, int* done,
                               cudaStream_t s) {
    if (c.n > kLuMaxN) return cudaErrorInvalidValue;
    const size_t smem = newton_lu32_smem_bytes(c.n);
    cudaError_t e = cudaFuncSetAttribute(k_newton_lu32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_newton_lu32<<<1, kLuT, smem, s>>>(c, J, As, rowinfo, F, xtab, coef, rho, stats, status, done);
    return cudaGetLastError();
}

}  // namespace dse
