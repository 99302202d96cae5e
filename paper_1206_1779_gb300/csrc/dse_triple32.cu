// dse_triple32.cu -- FP32-integrand variant of the quadrature kernel for the
// mixed-precision mode (precision = 1).
//
// Same data flow and outputs as k_triple in dse_triple.cu (Upart, Vpart in
// FP64, identical layouts), but every per-triple quantity -- z, s(z), T_j(s),
// ln G(z), ln Z(z), the exponentials, the kernels M and Q and the three
// integrands -- is evaluated in FP32, where this GPU has 64 times the FP64
// rate.  Accumulation is blocked: 32-term warp sums and BT-term tile sums in
// FP32, everything beyond a tile in FP64.  T_j(s) uses the forward recurrence
// rewritten in differences, D_{j+1} = sgn(s) (D_j - 2 (1 - |s|) T_j),
// T_{j+1} = sgn(s) T_j + D_{j+1}, whose rounding errors grow like j rather than
// j^2 near s = +-1.  The Jacobian built from these sums carries relative errors
// of ~1e-6; the mixed-precision Newton iteration pairs it with an FP64 residual.
#include "dse_internal.cuh"

namespace dse {

namespace {

constexpr unsigned kFullMask = 0xffffffffu;

__host__ __device__ inline int bt32_for(int N) { return N <= 96 ? 128 : 64; }

__host__ __device__ inline size_t tile32_floats(bool full, int N, int BT) {
    if (!full) return 0;
    const size_t t = (size_t)BT * (size_t)(N + 1);
    const int nact = N < BT ? N : BT;
    const size_t red = 2u * (size_t)(BT / nact) * 3u * (size_t)N;  // doubles as float pairs
    return t > red ? t : red;
}

__host__ __device__ inline size_t smem32_bytes(bool full, int N, int BT) {
    return tile32_floats(full, N, BT) * sizeof(float) + 3u * BT * sizeof(float) + 2u * N * sizeof(float);
}

template <int BT, int NJ, bool FULL>
__global__ void __launch_bounds__(BT) k_triple32(const __grid_constant__ TripleArgs A) {
    extern __shared__ __align__(16) float smem32[];
    const Consts& c = A.c;
    const int N = c.N;
    const int ldT = N + 1;
    float* sT = smem32;
    float* sh = smem32 + tile32_floats(FULL, N, BT);
    float* sa = sh + 3 * BT;
    float* sb = sa + N;
    constexpr int WARPS = BT / 32;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;

    // a (NZ) and b (NG) zero-padded to N = max(NZ, NG): one recurrence serves both series
    for (int j = tid; j < N; j += BT) {
        sa[j] = j < c.NZ ? (float)A.coef[j] : 0.0f;
        sb[j] = j < c.NG ? (float)A.coef[c.NZ + j] : 0.0f;
    }
    const int rt = blockIdx.y;
    const int ks = blockIdx.x;
    const Row row = A.rows[rt];
    const bool gluon = (row.flags & kRowGluon) != 0;
    const bool ghost = (row.flags & kRowGhost) != 0;
    const int k0 = ks * A.KB;
    const int k1 = min(c.nr, k0 + A.KB);
    const int nch = A.nch;
    const int nunits = k1 > k0 ? (k1 - k0) * nch : 0;
    const float L0 = (float)c.L0, invL1 = (float)c.invL1;
    const float eps2 = (float)c.eps2, lam2 = (float)c.lam2;
    const float ln_eps2 = (float)c.ln_eps2, ln_lam2 = (float)c.ln_lam2;
    const float kappa = (float)c.kappa, delta = (float)c.delta, gam = (float)c.gam;
    const float pG = (float)c.pG, qZ = (float)c.qZ, omega = (float)c.omega;
    const float sx = (float)row.sx;

    const int nact = N < BT ? N : BT;
    const int NG = BT / nact;
    const int g = tid / nact;
    const int jb = tid - g * nact;
    const bool bact = g < NG;
    const int mlo = (g * BT) / NG;
    const int mhi = ((g + 1) * BT) / NG;

    double acc[3][NJ];
#pragma unroll
    for (int jj = 0; jj < NJ; ++jj) acc[0][jj] = acc[1][jj] = acc[2][jj] = 0.0;

    __syncthreads();

    for (int base = 0; base < nunits; base += WARPS) {
        const int u = base + warp;
        float hQ = 0.0f, hM = 0.0f, hG = 0.0f;
        float* Trow = sT + (size_t)tid * ldT;
        bool live = false;
        int k = 0, ch = 0;
        if (u < nunits) {
            const int kk = u / nch;
            ch = u - kk * nch;
            k = k0 + kk;
            const int l = ch * 32 + lane;
            if (l < c.na) {
                live = true;
                const Rad rd = A.rad[rad_offset(c, rt) + k];
                const YTab yt = A.ytab[rad_offset(c, rt) + k];
                const Ang an = A.ang[l];
                const float sy = (float)rd.sy;
                const float sig = (float)an.sig;
                const float d0 = sx - sy;
                const float d = d0 * d0;
                const float b = 2.0f * sx * sy;
                const float z = fmaf(2.0f * b, sig, d);
                const float lz = logf(z);
                float s = (lz - L0) * invL1;
                s = fminf(1.0f, fmaxf(-1.0f, s));
                // T_0 = 1 (phi_0 = 1/2), T_1 = s, then the difference form
                float lg = 0.5f * sb[0];
                float lzz = 0.5f * sa[0];
                if (FULL) Trow[0] = 0.5f;
                if (N > 1) {
                    lg = fmaf(sb[1], s, lg);
                    lzz = fmaf(sa[1], s, lzz);
                    if (FULL) Trow[1] = s;
                }
                const float sg = s < 0.0f ? -1.0f : 1.0f;
                const float m2d = -2.0f * (1.0f - fabsf(s));
                float T = s;
                float D = s - sg;
                for (int j = 2; j < N; ++j) {
                    D = sg * fmaf(m2d, T, D);
                    T = fmaf(sg, T, D);
                    lg = fmaf(sb[j], T, lg);
                    lzz = fmaf(sa[j], T, lzz);
                    if (FULL) Trow[j] = T;
                }
                if (c.extrap == 0) {
                    if (z < eps2) {
                        const float r = lz - ln_eps2;
                        lg = fmaf(-kappa, r, lg);
                        lzz = fmaf(2.0f * kappa, r, lzz);
                    } else if (z > lam2) {
                        const float L = log1pf(omega * (lz - ln_lam2));
                        lg = fmaf(delta, L, lg);
                        lzz = fmaf(gam, L, lzz);
                    }
                }
                const float wgt = (float)(rd.W * an.w);
                const float iz = 1.0f / z;
                const float iz2 = iz * iz;
                const float s2 = (float)an.s2;
                if (ghost) {
                    const float Zz = expf(lzz);
                    hG = wgt * (float)yt.yG * (float)an.s4 * Zz * iz2;
                }
                if (gluon) {
                    const float Gz = expf(lg);
                    const float Wv = expf((float)yt.pq + pG * lg + qZ * lzz);
                    const float dd = d * d, db = d * b, bb = b * b;
                    const float n0 = 7.5f * dd;
                    const float n1 = -(48.0f * dd + 18.0f * db + 12.0f * bb);
                    const float n2 = 48.0f * dd - 48.0f * db - 38.0f * bb;
                    const float n3 = 96.0f * db + 64.0f * bb;
                    const float n4 = 16.0f * bb;
                    const float num = fmaf(sig, fmaf(sig, fmaf(sig, fmaf(sig, n4, n3), n2), n1), n0);
                    const float Q = 0.5f * num * iz2;
                    const float M = (float)rd.y * s2 * iz;
                    hQ = wgt * s2 * Q * Wv;
                    hM = wgt * s2 * M * (float)yt.G * Gz;
                }
            }
        }
        if (FULL && !live) {
            for (int j = 0; j < N; ++j) Trow[j] = 0.0f;
        }
        float rQ = hQ, rM = hM, rG = hG;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            rQ += __shfl_xor_sync(kFullMask, rQ, off);
            rM += __shfl_xor_sync(kFullMask, rM, off);
            rG += __shfl_xor_sync(kFullMask, rG, off);
        }
        if (u < nunits && lane == 0) {
            double* up = A.Upart + (((size_t)rt * c.nr + k) * nch + ch) * 3;
            up[0] = (double)rQ;
            up[1] = (double)rM;
            up[2] = (double)rG;
        }
        if (FULL) {
            sh[tid] = hQ;
            sh[BT + tid] = hM;
            sh[2 * BT + tid] = hG;
            __syncthreads();
            if (bact) {
                float t0[NJ], t1[NJ], t2[NJ];
#pragma unroll
                for (int jj = 0; jj < NJ; ++jj) t0[jj] = t1[jj] = t2[jj] = 0.0f;
                for (int m = mlo; m < mhi; ++m) {
                    const float q = sh[m];
                    const float mm = sh[BT + m];
                    const float gg = sh[2 * BT + m];
                    const float* Tm = sT + (size_t)m * ldT;
#pragma unroll
                    for (int jj = 0; jj < NJ; ++jj) {
                        const int j = jb + jj * nact;
                        if (j < N) {
                            const float t = Tm[j];
                            t0[jj] = fmaf(q, t, t0[jj]);
                            t1[jj] = fmaf(mm, t, t1[jj]);
                            t2[jj] = fmaf(gg, t, t2[jj]);
                        }
                    }
                }
                // tile sums join the FP64 accumulators
#pragma unroll
                for (int jj = 0; jj < NJ; ++jj) {
                    acc[0][jj] += (double)t0[jj];
                    acc[1][jj] += (double)t1[jj];
                    acc[2][jj] += (double)t2[jj];
                }
            }
            __syncthreads();
        }
    }

    if (FULL) {
        double* red = reinterpret_cast<double*>(sT);  // [NG][3][N]
        if (bact) {
#pragma unroll
            for (int jj = 0; jj < NJ; ++jj) {
                const int j = jb + jj * nact;
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

template <int BT, bool FULL>
cudaError_t launch32_bt(const TripleArgs& a, cudaStream_t s) {
    const int N = a.c.N;
    const size_t smem = smem32_bytes(FULL, N, BT);
    const dim3 grid(a.KS, a.Rt);
    const int nj = (N + BT - 1) / BT;
    cudaError_t e = cudaSuccess;
    if (nj <= 1) {
        e = cudaFuncSetAttribute(k_triple32<BT, 1, FULL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_triple32<BT, 1, FULL><<<grid, BT, smem, s>>>(a);
    } else if (nj <= 2) {
        e = cudaFuncSetAttribute(k_triple32<BT, 2, FULL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_triple32<BT, 2, FULL><<<grid, BT, smem, s>>>(a);
    } else if (nj <= 4) {
        e = cudaFuncSetAttribute(k_triple32<BT, 4, FULL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_triple32<BT, 4, FULL><<<grid, BT, smem, s>>>(a);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_triple32(bool full, const TripleArgs& a, cudaStream_t s) {
    if (a.KS <= 0 || a.Rt <= 0) return cudaSuccess;
    if (bt32_for(a.c.N) == 128) return full ? launch32_bt<128, true>(a, s) : launch32_bt<128, false>(a, s);
    return full ? launch32_bt<64, true>(a, s) : launch32_bt<64, false>(a, s);
}

}  // namespace dse
