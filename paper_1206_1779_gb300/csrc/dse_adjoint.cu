// dse_adjoint.cu -- derivative kernels for differentiating through the
// renormalised ghost-gluon system F(c; g^2 Nc, G(x_G)^{-1}, Z(x_Z)^{-1}) of
// arXiv:1206.1779 Sec. 2-3:
//   * the vector-Jacobian product v^T dF/dc contracted from the per-row
//     derivative sums D (the Newton matrix itself is never formed);
//   * dF/d(g^2 Nc, G(x_G)^{-1}, Z(x_Z)^{-1}): the coupling enters through the
//     prefactor K = g^2 Nc/(2 pi)^3 of both self-energies and through
//     omega = 11 g^2 Nc/(48 pi^2) of the UV forms of G(z), Z(z) (Sec. 2), the two
//     boundary values enter the MOM-subtracted rows with coefficient -1;
//   * power-of-two row equilibration and an in-place transpose for the adjoint
//     system J^T lambda = g;
//   * the vector-Jacobian product of ln G(x), ln Z(x) (Sec. 3 expansion with the
//     Sec. 2 IR/UV continuation) with respect to c and g^2 Nc.
#include "dse_internal.cuh"

namespace dse {

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kParamThreads = 256;
constexpr int kVjpThreads = 128;
constexpr int kDvThreads = 256;  // 32 coefficients x 8 point lanes

// d omega / d(g^2 Nc)
__device__ __forceinline__ double domega() { return 11.0 / (48.0 * kPi * kPi); }

// Per row r (0..Rc-1 collocation, Rc: x_Z, Rc+1: x_G) the omega-weighted sums
//   wZ = sum hQ (p dlnG/dw + q dlnZ/dw)(z) + hM dlnG/dw(z)   (gluon rows)
//   wG = sum hG dlnZ/dw(z)                                   (ghost rows)
// over the triples with z > lambda2, where ln G(z) = ln G(lambda2) + delta L,
// ln Z(z) = ln Z(lambda2) + gamma L, L = ln(1 + omega ln(z/lambda2)) and
// d ln G/d omega = delta l/(1 + omega l), l = ln(z/lambda2).  Then
//   dPi_Z/dg = Pi_Z/g + K/(3x) omega' wZ,   dPi_G/dg = Pi_G/g - K omega' wG,
// with Pi from the residual pass (D[r][2n], D[r][2n+1]).  Fixed-order
// reductions: thread-strided sums, warp shuffles, then warps in order.
__global__ void __launch_bounds__(kParamThreads) k_param_rows(const Consts c, const Rad* __restrict__ rad,
                                                               const Ang* __restrict__ ang,
                                                               const Row* __restrict__ rows,
                                                               const YTab* __restrict__ ytab,
                                                               const double* __restrict__ coef,
                                                               const double* __restrict__ D, double g2nc,
                                                               double* __restrict__ dPi) {
    __shared__ double s_w[2][kParamThreads / 32];
    const int NZ = c.NZ, NG = c.NG, n = c.n, Rc = c.Rc;
    const int r = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool special = (r == Rc + 1) && !(c.x_G > 0.0);  // x_G = 0: z = y <= lambda2
    const int flags = special ? kRowGhost : rows[r].flags;
    const bool gluon = (flags & kRowGluon) != 0;
    const bool ghost = (flags & kRowGhost) != 0;
    double wZ = 0.0, wG = 0.0;
    if (!special && c.extrap == 0) {
        const Row row = rows[r];
        // Chebyshev part at s = 1: T_j(1) = 1, phi_0 = 1/2
        double lZb = 0.5 * coef[0], lGb = 0.5 * coef[NZ];
        for (int j = 1; j < NZ; ++j) lZb += coef[j];
        for (int j = 1; j < NG; ++j) lGb += coef[NZ + j];
        const int total = c.nr * c.na;
        for (int t = tid; t < total; t += kParamThreads) {
            const int k = t / c.na;
            const int l = t - k * c.na;
            const Rad rd = rad[rad_offset(c, r) + k];
            const Ang an = ang[l];
            const double d0 = row.sx - rd.sy;
            const double d = d0 * d0;
            const double b = 2.0 * row.sx * rd.sy;
            const double z = fma(2.0 * b, an.sig, d);
            if (!(z > c.lam2)) continue;
            const YTab yt = ytab[rad_offset(c, r) + k];
            const double lu = log(z) - c.ln_lam2;
            const double den = 1.0 / fma(c.omega, lu, 1.0);
            const double L = log1p(c.omega * lu);
            const double lg = fma(c.delta, L, lGb);
            const double lzz = fma(c.gam, L, lZb);
            const double gw = c.delta * lu * den;
            const double zw = c.gam * lu * den;
            const double wgt = rd.W * an.w;
            const double iz = 1.0 / z;
            const double iz2 = iz * iz;
            if (ghost) {
                const double hG = wgt * yt.yG * an.s4 * exp(lzz) * iz2;
                wG = fma(hG, zw, wG);
            }
            if (gluon) {
                const double Wv = exp(yt.pq + c.pG * lg + c.qZ * lzz);
                const double dd = d * d, db = d * b, bb = b * b;
                const double n0 = 7.5 * dd;
                const double n1 = -(48.0 * dd + 18.0 * db + 12.0 * bb);
                const double n2 = 48.0 * dd - 48.0 * db - 38.0 * bb;
                const double n3 = 96.0 * db + 64.0 * bb;
                const double n4 = 16.0 * bb;
                const double sg = an.sig;
                const double num = fma(sg, fma(sg, fma(sg, fma(sg, n4, n3), n2), n1), n0);
                const double Q = 0.5 * num * iz2;
                const double M = rd.y * an.s2 * iz;
                const double hQ = wgt * an.s2 * Q * Wv;
                const double hM = wgt * an.s2 * M * yt.G * exp(lg);
                wZ = fma(hQ, fma(c.pG, gw, c.qZ * zw), wZ);
                wZ = fma(hM, gw, wZ);
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        wZ += __shfl_xor_sync(kFullMask, wZ, off);
        wG += __shfl_xor_sync(kFullMask, wG, off);
    }
    if (lane == 0) {
        s_w[0][warp] = wZ;
        s_w[1][warp] = wG;
    }
    __syncthreads();
    if (tid == 0) {
        double tZ = 0.0, tG = 0.0;
        for (int w = 0; w < kParamThreads / 32; ++w) {
            tZ += s_w[0][w];
            tG += s_w[1][w];
        }
        const double* Dr = D + (size_t)r * ldD(c);
        const double pre = (gluon && !special) ? rows[r].pre : 0.0;
        dPi[2 * r] = gluon ? Dr[2 * n] / g2nc + pre * domega() * tZ : 0.0;
        dPi[2 * r + 1] = ghost ? Dr[2 * n + 1] / g2nc - c.K * domega() * tG : 0.0;
    }
}

// dF (n x 3, columns g^2 Nc, G(x_G)^{-1}, Z(x_Z)^{-1}) from the per-row dPi/dg
// (gluon rows i < NZ at row i, ghost rows i < NG at row gofs + i):
//   dF_z,i/dg = -dPi_Z(x_i)/dg + dPi_Z(x_Z)/dg,   dF_z,i/dZinv = -1
//   dF_g,i/dg = -dPi_G(x_i)/dg + dPi_G(x_G)/dg,   dF_g,i/dGinv = -1
// and optionally w = v^T dF (3 values, fixed-order sums by one warp).
__global__ void k_param_assemble(const Consts c, const double* __restrict__ dPi, double* __restrict__ dF,
                                 const double* __restrict__ v, double* __restrict__ vdF) {
    const int NZ = c.NZ, n = c.n, Rc = c.Rc;
    const int tid = threadIdx.x;
    if (dF) {
        for (int i = tid; i < n; i += blockDim.x) {
            double d0, d1, d2;
            if (i < NZ) {
                d0 = -dPi[2 * i] + dPi[2 * Rc];
                d1 = 0.0;
                d2 = -1.0;
            } else {
                const int r = c.gofs + (i - NZ);
                d0 = -dPi[2 * r + 1] + dPi[2 * (Rc + 1) + 1];
                d1 = -1.0;
                d2 = 0.0;
            }
            dF[(size_t)i * 3 + 0] = d0;
            dF[(size_t)i * 3 + 1] = d1;
            dF[(size_t)i * 3 + 2] = d2;
        }
    }
    if (v && tid < 32) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int i = tid; i < n; i += 32) {
            if (i < NZ) {
                a0 = fma(v[i], -dPi[2 * i] + dPi[2 * Rc], a0);
                a2 -= v[i];
            } else {
                const int r = c.gofs + (i - NZ);
                a0 = fma(v[i], -dPi[2 * r + 1] + dPi[2 * (Rc + 1) + 1], a0);
                a1 -= v[i];
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            a0 += __shfl_xor_sync(kFullMask, a0, off);
            a1 += __shfl_xor_sync(kFullMask, a1, off);
            a2 += __shfl_xor_sync(kFullMask, a2, off);
        }
        if (tid == 0) {
            vdF[0] = a0;
            vdF[1] = a1;
            vdF[2] = a2;
        }
    }
}

// out_j = sum_i v_i J[i][j] with the entries of J taken from the per-row
// derivative vectors as the assembly does (Sec. 3 matrix layout), one thread
// per column j, gluon rows then ghost rows in order.
__global__ void __launch_bounds__(kVjpThreads) k_vjp(const Consts c, const XTab* __restrict__ xtab,
                                                      const double* __restrict__ phix,
                                                      const double* __restrict__ D,
                                                      const double* __restrict__ v, double* __restrict__ out,
                                                      int* __restrict__ status) {
    const int N = c.N, NZ = c.NZ, NG = c.NG, n = c.n;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const size_t ld = ldD(c);
    const double* DZ = D + (size_t)c.Rc * ld;
    const double* DG = D + (size_t)(c.Rc + 1) * ld;
    double acc = 0.0;
    for (int i = 0; i < NZ; ++i) {
        const double* Di = D + (size_t)i * ld;
        const double diag = j < NZ ? -xtab[i].Zinv * phix[(size_t)i * N + j] : 0.0;
        acc = fma(v[i], diag - Di[j] + DZ[j], acc);
    }
    for (int i = 0; i < NG; ++i) {
        const int r = c.gofs + i;
        const double* Di = D + (size_t)r * ld;
        const double diag = j >= NZ ? -xtab[r].Ginv * phix[(size_t)r * N + (j - NZ)] : 0.0;
        acc = fma(v[NZ + i], diag - Di[n + j] + DG[n + j], acc);
    }
    out[j] = acc;
    if (!isfinite(acc)) atomicOr(status, kStatusNonfinite);
}

// A <- A^T for an n x n row-major matrix: the thread of entry (i, j), i < j,
// swaps it with (j, i); every pair has exactly one owner.
__global__ void k_transpose_inplace(int n, double* __restrict__ A) {
    const size_t total = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n);
        const int j = (int)(e % n);
        if (i < j) {
            const double a = A[e];
            const size_t et = (size_t)j * n + i;
            A[e] = A[et];
            A[et] = a;
        }
    }
}

// Row equilibration by exact powers of two before the transpose: J^T lambda = g
// is solved as (S J)^T mu = g, lambda = S mu, S = diag(2^(1022 - E_i)) with E_i
// the largest biased exponent in row i, so that the rows of the transposed
// system (the columns of S J) carry comparable magnitudes -- the rows of J span
// many decades (Z(x)^{-1} and the self-energies at the collocation points).
// One block per row; a zero row keeps scale 1 (the solver reports it singular).
__global__ void __launch_bounds__(128) k_row_equilibrate(int n, double* __restrict__ A, double* __restrict__ scale) {
    __shared__ int s_e[4];
    const int i = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double* row = A + (size_t)i * n;
    int e = 0;
    for (int j = tid; j < n; j += 128) e = max(e, (__double2hiint(row[j]) >> 20) & 0x7ff);
    e = __reduce_max_sync(kFullMask, e);
    if (lane == 0) s_e[warp] = e;
    __syncthreads();
    const int E = max(max(s_e[0], s_e[1]), max(s_e[2], s_e[3]));
    const double sc = (E > 0 && E < 0x7ff) ? __hiloint2double((1022 - E + 1023) << 20, 0) : 1.0;
    for (int j = tid; j < n; j += 128) row[j] *= sc;
    if (tid == 0) scale[i] = sc;
}

// lambda = S mu in place, and ||lambda||_inf into stats[2] (one block).
__global__ void __launch_bounds__(256) k_adjoint_finish(int n, const double* __restrict__ scale,
                                                        double* __restrict__ lam, double* __restrict__ stats) {
    __shared__ double s_m[8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double m = 0.0;
    for (int i = tid; i < n; i += 256) {
        const double v = lam[i] * scale[i];
        lam[i] = v;
        m = fmax(m, fabs(v));
    }
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(kFullMask, m, off));
    if (lane == 0) s_m[warp] = m;
    __syncthreads();
    if (tid == 0) {
        double t = s_m[0];
        for (int w = 1; w < 8; ++w) t = fmax(t, s_m[w]);
        stats[2] = t;
    }
}

// Vector-Jacobian product of the dressing functions at n points:
//   out[j]      = sum_m gZ_m d ln Z(x_m)/d a_j = sum_m gZ_m phi_j(x_m)   (j < NZ)
//   out[NZ + j] = sum_m gG_m d ln G(x_m)/d b_j = sum_m gG_m phi_j(x_m)   (j < NG)
//   out[n]      = sum_m (gG_m delta + gZ_m gamma) l_m/(1 + omega l_m) omega'
//                over x_m > lambda2 (UV form, the only place g^2 Nc enters)
// with phi_j(x) = 1/2 (j = 0), T_j(s(x)) and s clamped to [-1, 1] as in the
// expansion itself (the IR/UV forms add no coefficient dependence).
// Grid (coefficient block of 32, point split); thread (lane j, point lane p)
// runs the Chebyshev recurrence to its own j (j < N).  Partial sums [split][n+1].
__global__ void __launch_bounds__(kDvThreads) k_dressing_vjp_part(const Consts c, int n,
                                                                   const double* __restrict__ x,
                                                                   const double* __restrict__ gG,
                                                                   const double* __restrict__ gZ,
                                                                   double* __restrict__ part,
                                                                   int* __restrict__ status) {
    __shared__ double s_a[8][32], s_b[8][32], s_u[8][32];
    const int N = c.N;
    const int lane = threadIdx.x & 31;
    const int p = threadIdx.x >> 5;
    const int j = blockIdx.x * 32 + lane;
    const int split = blockIdx.y;
    const int nsplit = gridDim.y;
    const int m0 = (int)(((long long)n * split) / nsplit);
    const int m1 = (int)(((long long)n * (split + 1)) / nsplit);
    double sa = 0.0, sb = 0.0, su = 0.0;
    bool bad = false;
    for (int m = m0 + p; m < m1; m += 8) {
        const double xm = x[m];
        if (!(xm > 0.0)) {
            bad = true;
            continue;
        }
        const double lx = log(xm);
        double s = (lx - c.L0) * c.invL1;
        s = fmin(1.0, fmax(-1.0, s));
        if (j < N) {
            double t;
            if (j == 0) t = 0.5;
            else {
                double t0 = 1.0, t1 = s;
                const double s2 = 2.0 * s;
                for (int q = 2; q <= j; ++q) {
                    const double t2 = fma(s2, t1, -t0);
                    t0 = t1;
                    t1 = t2;
                }
                t = t1;
            }
            if (j < c.NZ) sa = fma(gZ[m], t, sa);
            if (j < c.NG) sb = fma(gG[m], t, sb);
        }
        if (j == 0 && c.extrap == 0 && xm > c.lam2) {
            const double lu = lx - c.ln_lam2;
            const double f = lu / fma(c.omega, lu, 1.0) * domega();
            su = fma(fma(gG[m], c.delta, gZ[m] * c.gam), f, su);
        }
    }
    s_a[p][lane] = sa;
    s_b[p][lane] = sb;
    s_u[p][lane] = su;
    __syncthreads();
    if (p == 0) {
        double ta = 0.0, tb = 0.0, tu = 0.0;
        for (int q = 0; q < 8; ++q) {
            ta += s_a[q][lane];
            tb += s_b[q][lane];
            tu += s_u[q][lane];
        }
        double* out = part + (size_t)split * (c.n + 1);
        if (j < c.NZ) out[j] = ta;
        if (j < c.NG) out[c.NZ + j] = tb;
        if (j == 0) out[c.n] = tu;
    }
    if (bad) atomicOr(status, kStatusNonfinite);
}

__global__ void k_dressing_vjp_reduce(int n, int nsplit, const double* __restrict__ part, double* __restrict__ out,
                                      double* __restrict__ out_g2nc) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e > n) return;
    double s = 0.0;
    for (int q = 0; q < nsplit; ++q) s += part[(size_t)q * (n + 1) + e];
    if (e < n) out[e] = s;
    else if (out_g2nc) *out_g2nc = s;
}

// Finite-difference Newton matrix (Sec. 4.2, the paper's Jacobian): the 2n
// perturbed coefficient vectors c +- h_j e_j, h_j = rel max(|c_j|, 1e-3), stored
// as vector v = 2 j (+) and 2 j + 1 (-), n entries each.
__global__ void k_fd_perturb(int n, const double* __restrict__ coef, double rel, double* __restrict__ out) {
    const size_t total = 2 * (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int v = (int)(e / n);
        const int i = (int)(e - (size_t)v * n);
        const int j = v >> 1;
        double x = coef[i];
        if (i == j) {
            const double h = rel * fmax(fabs(x), 1e-3);
            x = (v & 1) ? x - h : x + h;
        }
        out[e] = x;
    }
}

// J[i][j] = (F(c + h e_j)_i - F(c - h e_j)_i) / ((c_j + h) - (c_j - h)), the
// denominator taken from the perturbed values actually used.
__global__ void k_fd_columns(int n, const double* __restrict__ pert, const double* __restrict__ Fall,
                             double* __restrict__ J, int* __restrict__ status) {
    const size_t total = (size_t)n * n;
    bool bad = false;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n);
        const int j = (int)(e - (size_t)i * n);
        const size_t vp = 2 * (size_t)j * n, vm = vp + n;
        const double v = (Fall[vp + i] - Fall[vm + i]) / (pert[vp + j] - pert[vm + j]);
        J[e] = v;
        bad |= !isfinite(v);
    }
    if (bad) atomicOr(status, kStatusNonfinite);
}

// Row prefactors K/(3x) after a change of g^2 Nc.
__global__ void k_row_prefactors(const Consts c, Row* __restrict__ rows, int Rt) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Rt) return;
    const double x = rows[q].x;
    rows[q].pre = x > 0.0 ? c.K / (3.0 * x) : 0.0;
}

int blocks_for(long long total, int threads) {
    long long b = (total + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 4096) b = 4096;
    return (int)b;
}

}  // namespace

cudaError_t launch_param_derivatives(const Consts& c, const Rad* rad, const Ang* ang, const Row* rows,
                                     const YTab* ytab, const double* coef, const double* D, double g2nc,
                                     double* dPi, double* dF, const double* v, double* vdF, cudaStream_t s) {
    k_param_rows<<<c.Rc + 2, kParamThreads, 0, s>>>(c, rad, ang, rows, ytab, coef, D, g2nc, dPi);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_param_assemble<<<1, 256, 0, s>>>(c, dPi, dF, v, vdF);
    return cudaGetLastError();
}

cudaError_t launch_vjp(const Consts& c, const XTab* xtab, const double* phix, const double* D, const double* v,
                       double* out, int* status, cudaStream_t s) {
    k_vjp<<<(c.n + kVjpThreads - 1) / kVjpThreads, kVjpThreads, 0, s>>>(c, xtab, phix, D, v, out, status);
    return cudaGetLastError();
}

cudaError_t launch_equilibrate_transpose(int n, double* A, double* scale, cudaStream_t s) {
    k_row_equilibrate<<<n, 128, 0, s>>>(n, A, scale);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_transpose_inplace<<<blocks_for((long long)n * n, 256), 256, 0, s>>>(n, A);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_finish(int n, const double* scale, double* lam, double* stats, cudaStream_t s) {
    k_adjoint_finish<<<1, 256, 0, s>>>(n, scale, lam, stats);
    return cudaGetLastError();
}

int dressing_vjp_splits(int n) {
    int q = (n + 255) / 256;
    if (q < 1) q = 1;
    if (q > kDressingVjpMaxSplits) q = kDressingVjpMaxSplits;
    return q;
}

cudaError_t launch_dressing_vjp(const Consts& c, int n, const double* x, const double* gG, const double* gZ,
                                double* part, int nsplit, double* out, double* out_g2nc, int* status,
                                cudaStream_t s) {
    const dim3 grid((c.N + 31) / 32, nsplit);
    k_dressing_vjp_part<<<grid, kDvThreads, 0, s>>>(c, n, x, gG, gZ, part, status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_dressing_vjp_reduce<<<(c.n + 1 + 127) / 128, 128, 0, s>>>(c.n, nsplit, part, out, out_g2nc);
    return cudaGetLastError();
}

cudaError_t launch_fd_perturb(int n, const double* coef, double rel, double* out, cudaStream_t s) {
    k_fd_perturb<<<blocks_for(2LL * n * n, 256), 256, 0, s>>>(n, coef, rel, out);
    return cudaGetLastError();
}

cudaError_t launch_fd_columns(int n, const double* pert, const double* Fall, double* J, int* status, cudaStream_t s) {
    k_fd_columns<<<blocks_for((long long)n * n, 256), 256, 0, s>>>(n, pert, Fall, J, status);
    return cudaGetLastError();
}

cudaError_t launch_row_prefactors(const Consts& c, Row* rows, int Rt, cudaStream_t s) {
    k_row_prefactors<<<(Rt + 127) / 128, 128, 0, s>>>(c, rows, Rt);
    return cudaGetLastError();
}

}  // namespace dse
