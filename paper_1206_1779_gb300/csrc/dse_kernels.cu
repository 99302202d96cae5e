// dse_kernels.cu -- set-up, table, contraction, assembly, Newton-step and
// Schwinger-function kernels of the sm_103a solver (arXiv:1206.1779).
#include "dse_df.cuh"
#include "dse_internal.cuh"
#include "dse_series.cuh"

namespace dse {

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr unsigned kFullMask = 0xffffffffu;

// ------------------------------------------------------------------------
// Gauss-Legendre rule (Sec. 2 radial/angular rules; Sec. 5 node generation
// in parallel): one thread per root pair, Newton iteration on the three-term
// Legendre recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}, starting from
// cos(pi (i + 3/4)/(n + 1/2)); the weight 2 / ((1 - x^2) P_n'(x)^2) is taken
// from one more recurrence pass at the converged root.
__device__ __forceinline__ void legendre_pair(int n, double r, const double* __restrict__ inv, double& pn,
                                              double& pnm1) {
    double p0 = 1.0, p1 = r;
    for (int k = 1; k < n; ++k) {
        const double rp1 = r * p1;
        // p2 = ((2k+1) r p1 - k p0) / (k+1) = r p1 + (r p1 - p0) k/(k+1)
        const double p2 = fma(rp1 - p0, (double)k * inv[k + 1], rp1);
        p0 = p1;
        p1 = p2;
    }
    pn = p1;
    pnm1 = p0;
}

__global__ void k_inverse_table(int n, double* inv) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k <= n) inv[k] = k > 0 ? 1.0 / (double)k : 0.0;
}

__global__ void k_gauss_legendre(int n, const double* __restrict__ inv, double* __restrict__ x,
                                 double* __restrict__ w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int half = (n + 1) / 2;
    if (i >= half) return;
    double r = cos(kPi * ((double)i + 0.75) / ((double)n + 0.5));
    double pn, pm;
    for (int it = 0; it < 100; ++it) {
        legendre_pair(n, r, inv, pn, pm);
        const double dp = (double)n * (r * pn - pm) / (r * r - 1.0);
        const double dr = pn / dp;
        r -= dr;
        if (fabs(dr) <= 1e-16 * (1.0 + fabs(r))) break;
    }
    legendre_pair(n, r, inv, pn, pm);
    const double dp = (double)n * (r * pn - pm) / (r * r - 1.0);
    const double wt = 2.0 / ((1.0 - r * r) * dp * dp);
    const int hi = n - 1 - i;
    x[hi] = r;
    w[hi] = wt;
    if (i != hi) {
        x[i] = -r;
        w[i] = wt;
    }
}

// Mapped rules: radial t = ln y = L0 + L1 tau (weight L1 omega y), angular
// theta = pi/2 (1 + tau) (weight pi/2 omega), collocation points at the mapped
// roots s_i = -cos(pi (2i+1)/(2m)) of T_m (Sec. 3; m = NZ for the gluon rows,
// NG for the ghost rows, one shared set when NZ = NG), triple-kernel rows.
__device__ __forceinline__ double collocation_point(const Consts& c, int q) {
    const int m = q < c.NZ ? c.NZ : c.NG;
    const int i = q < c.NZ ? q : q - c.NZ;
    const double s = -cos(kPi * (2.0 * i + 1.0) / (2.0 * m));
    return exp(c.L0 + c.L1 * s);
}

__global__ void k_setup_rules(const Consts c, const double* __restrict__ gr, const double* __restrict__ wr,
                              const double* __restrict__ ga, const double* __restrict__ wa, Rad* __restrict__ rad,
                              Ang* __restrict__ ang, double* __restrict__ theta, double* __restrict__ xcol,
                              Row* __restrict__ rows, int Rt) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int nrad = (int)rad_entries(c);
    if (m < nrad) {
        Rad r;
        if (c.radmode == 0) {
            const double y = exp(c.L0 + c.L1 * gr[m]);
            r.y = y;
            r.W = c.L1 * wr[m] * y;
        } else {
            // row rr's split rule: [1e-6 eps2, eps2], [eps2, x], [x, lambda2] in ln y,
            // x clamped into [eps2, lambda2]; nrule Gauss-Legendre nodes per piece
            const int rr = m / c.nr;
            const int k = m - rr * c.nr;
            const int piece = k / c.nrule;
            const int i = k - piece * c.nrule;
            double x = rr < c.Rc ? collocation_point(c, rr) : (rr == c.Rc ? c.x_Z : c.x_G);
            x = fmin(fmax(x, c.eps2), c.lam2);
            const double lx = log(x);
            const double lo = piece == 0 ? c.ln_eps2 + log(1e-6) : (piece == 1 ? c.ln_eps2 : lx);
            const double hi = piece == 0 ? c.ln_eps2 : (piece == 1 ? lx : c.ln_lam2);
            const double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
            const double y = exp(mid + half * gr[i]);
            r.y = y;
            r.W = half * wr[i] * y;
        }
        r.sy = sqrt(r.y);
        r.pad = 0.0;
        rad[m] = r;
        return;
    }
    int q = m - nrad;
    if (q < c.na) {
        Ang a;
        double th;
        if (c.angmode == 0) {
            th = 0.5 * kPi * (1.0 + ga[q]);
            const double sh = sin(0.5 * th);
            const double sn = sin(th);
            a.w = 0.5 * kPi * wa[q];
            a.sig = sh * sh;
            a.s2 = sn * sn;
        } else {
            // tanh-sinh in xi = cos theta = tanh u, u = (pi/2) sinh t, t = t_max - (q + 1/2) h:
            // sin^2(theta/2) = 1/(1 + e^{2u}), sin^2 theta = 1/cosh^2 u, theta = 2 atan(e^{-u}),
            // weight (pi/2) h cosh t / cosh u
            const double tmax = 4.0;
            const double h = 2.0 * tmax / c.na;
            const double t = tmax - (q + 0.5) * h;
            const double u = 0.5 * kPi * sinh(t);
            const double cu = cosh(u);
            th = 2.0 * atan(exp(-u));
            a.w = h * 0.5 * kPi * cosh(t) / cu;
            a.sig = 1.0 / (1.0 + exp(2.0 * u));
            a.s2 = 1.0 / (cu * cu);
        }
        a.s4 = a.s2 * a.s2;
        a.ws2 = a.w * a.s2;
        a.ws4 = a.w * a.s4;
        ang[q] = a;
        theta[q] = th;
        return;
    }
    q -= c.na;
    if (q < c.Rc) {
        xcol[q] = collocation_point(c, q);
        return;
    }
    q -= c.Rc;
    if (q < Rt) {
        double x;
        int flags;
        if (q < c.Rc) {
            x = collocation_point(c, q);
            flags = c.gofs == 0 ? (kRowGluon | kRowGhost) : (q < c.NZ ? kRowGluon : kRowGhost);
        } else if (q == c.Rc) {
            x = c.x_Z;
            flags = kRowGluon;
        } else {
            x = c.x_G;
            flags = kRowGhost;
        }
        Row r;
        r.x = x;
        r.sx = sqrt(x);
        r.pre = x > 0.0 ? c.K / (3.0 * x) : 0.0;
        r.flags = flags;
        r.pad = 0;
        rows[q] = r;
    }
}

// Dressing functions at the radial nodes and collocation points for the
// current coefficients, with the basis tables phi_j(y_k), phi_j(x_i).
__device__ __forceinline__ void tables_unit(const Consts& c, const double* __restrict__ coef, const Rad* __restrict__ rad,
                         const double* __restrict__ xcol, YTab* __restrict__ ytab, double* __restrict__ phiy,
                         XTab* __restrict__ xtab, double* __restrict__ phix, const int m) {
    const double* a = coef;
    const double* b = coef + c.NZ;
    const int nrad = (int)rad_entries(c);
    if (m < nrad) {
        const double y = rad[m].y;
        double lG, lZ;
        dressing_eval(c, a, b, y, lG, lZ, phiy + (size_t)m * c.N);
        YTab t;
        t.lG = lG;
        t.lZ = lZ;
        t.G = exp(lG);
        t.Z = exp(lZ);
        t.pq = c.pG * lG + c.qZ * lZ;
        t.yG = y * t.G;
        t.Wy = exp(t.pq);
        t.pad1 = 0.0;
        ytab[m] = t;
        return;
    }
    const int i = m - nrad;
    if (i < c.Rc) {
        double lG, lZ;
        dressing_eval(c, a, b, xcol[i], lG, lZ, phix + (size_t)i * c.N);
        XTab t;
        t.lG = lG;
        t.lZ = lZ;
        t.G = exp(lG);
        t.Z = exp(lZ);
        t.Ginv = exp(-lG);
        t.Zinv = exp(-lZ);
        t.pad0 = t.pad1 = 0.0;
        xtab[i] = t;
    }
}

__global__ void k_tables(const Consts c, const double* __restrict__ coef, const Rad* __restrict__ rad,
                         const double* __restrict__ xcol, YTab* __restrict__ ytab, double* __restrict__ phiy,
                         XTab* __restrict__ xtab, double* __restrict__ phix) {
    tables_unit(c, coef, rad, xcol, ytab, phiy, xtab, phix, blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void k_tables_batched(const BatchProblem* __restrict__ P, const double* __restrict__ coef_base) {
    const BatchProblem& B = P[blockIdx.y];
    if (!B.active) return;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= (int)rad_entries(B.t.c) + B.t.c.Rc) return;
    tables_unit(B.t.c, coef_base + B.coef_off, B.t.rad, B.xcol, B.ytab, B.phiy, B.xtab, B.phix, m);
}

// ------------------------------------------------------------------------
// Series table (see SeriesRec).  Error-free transformations for the node values:
// TwoSum (Knuth) and the FMA form of TwoProduct give exact rounding errors; a
// double-double value is hi + lo with |lo| <= ulp(hi)/2.
struct DD { double hi, lo; };

__device__ __forceinline__ DD dd_two_sum(double a, double b) {
    const double s = a + b;
    const double bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ DD dd_fast_two_sum(double a, double b) {  // |a| >= |b|
    const double s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ DD dd_add(DD x, DD y) {
    DD s = dd_two_sum(x.hi, y.hi);
    const DD t = dd_two_sum(x.lo, y.lo);
    s.lo += t.hi;
    s = dd_fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return dd_fast_two_sum(s.hi, s.lo);
}

// c_0/2 + sum_{j>=1} c_j T_j(s) at s = s_h + s_l (a double-double node) by the
// compensated Clenshaw recurrence: b_k = c_k + 2 s b_{k+1} - b_{k+2} in FP64, the
// exact rounding error of every step from TwoProduct / TwoSum, and those errors
// carried through the same linear recurrence in FP64; the sum of both is the
// series as computed in about twice the working precision, rounded once.
// cf: the coefficients in shared memory.
__device__ double series_comp(const double* cf, int m, double sh, double sl) {
    const double s2h = 2.0 * sh, s2l = 2.0 * sl;
    double b1 = 0.0, b2 = 0.0, e1 = 0.0, e2 = 0.0;
    for (int k = m - 1; k >= 1; --k) {
        const double p = s2h * b1;
        const double ep = fma(s2h, b1, -p);
        const DD q = dd_two_sum(p, -b2);
        const DD t = dd_two_sum(q.hi, cf[k]);
        const double local = (ep + q.lo) + fma(s2l, b1, t.lo);
        const double ek = fma(s2h, e1, local - e2);
        b2 = b1;
        b1 = t.hi;
        e2 = e1;
        e1 = ek;
    }
    const double p = sh * b1;
    const double ep = fma(sh, b1, -p);
    const DD q = dd_two_sum(p, -b2);
    const DD t = dd_two_sum(q.hi, 0.5 * cf[0]);
    const double local = (ep + q.lo) + fma(sl, b1, t.lo);
    return t.hi + fma(sh, e1, local - e2);
}

// The interval geometry of the table: mid = (cos th0 + cos th1)/2 and
// half = (cos th0 - cos th1)/2 = sin((th0 + th1)/2) sin(h/2) (no cancellation) of
// interval i, th0 = i h, th1 = (i + 1) h, h = pi/M; and the node
// s = mid + half u_q at the q-th Chebyshev point u_q = cos(pi (q + 1/2)/Q), held
// exactly as a double-double.
__device__ __forceinline__ void series_interval(const int M, const int i, double& mid, double& half) {
    const double h = kPi / M;
    const double th0 = i * h, th1 = (i + 1) * h;
    double s0, c0, s1, c1, sm, cm, sh, ch;
    sincos(th0, &s0, &c0);
    sincos(th1, &s1, &c1);
    sincos(0.5 * (th0 + th1), &sm, &cm);
    sincos(0.5 * h, &sh, &ch);
    mid = 0.5 * (c0 + c1);
    half = sm * sh;
}

__device__ __forceinline__ DD series_node(const double mid, const double half, const int q) {
    const double uq = cos(kPi * (q + 0.5) / kSeriesQ);
    const DD p = dd_two_sum(half * uq, mid);
    return dd_add(p, DD{fma(half, uq, -(half * uq)), 0.0});
}

// The interpolation table dct[k][r] = cos(pi k (r + 1/2)/Q) (one entry per call)
// and, by lanes 0 .. Q-1 of a warp together, the monomial coefficients
// tcoef[j][k] = [u^k] T_j(u) by the three-term recurrence (exact integers).
__device__ __forceinline__ void series_tcoef_column(const int k, double (*tcoef)[kSeriesQ]) {
    double tm = k == 0 ? 1.0 : 0.0;  // T_0
    double tc = k == 1 ? 1.0 : 0.0;  // T_1
    tcoef[0][k] = tm;
    tcoef[1][k] = tc;
    for (int j = 2; j < kSeriesQ; ++j) {
        const double lower = __shfl_up_sync(0x0000ffffu, tc, 1);  // [u^{k-1}] T_{j-1}
        const double tn = (k == 0 ? 0.0 : 2.0 * lower) - tm;
        tcoef[j][k] = tn;
        tm = tc;
        tc = tn;
    }
}

// The end-point record: sum_j c_j T_j(+-1) with T_j(1) = 1, T_j(-1) = (-1)^j, in
// the order of the per-triple recurrence (e: 0 ln Z(1), 1 ln G(1), 2 ln Z(-1),
// 3 ln G(-1)).
__device__ __forceinline__ void series_endpoint(const Consts& c, const double* cf_ab, const int e, SeriesRec* tab) {
    const int nc = (e & 1) ? c.NG : c.NZ;
    const double* cf = cf_ab + ((e & 1) ? c.NZ : 0);
    const double sgn = e < 2 ? 1.0 : -1.0;
    double v = 0.5 * cf[0];
    double t = 1.0;
    for (int j = 1; j < nc; ++j) {
        t *= sgn;
        v = fma(cf[j], t, v);
    }
    reinterpret_cast<double*>(tab + kSeriesM)[e] = v;
}

// From the node values ln Z, ln G of IPB intervals (sv[f][il][q]) to their records:
// thread (f, il, q) forms the node value F (0: Z = e^{ln Z}, 1: G = e^{ln G},
// 2: W = e^{p ln G + q ln Z}), the Chebyshev coefficient of degree q of F's
// interpolant, c_q = (2 - [q = 0])/Q sum_r v_r cos(pi q (r + 1/2)/Q), and its
// monomial coefficient of u^q, sum_j c_j [u^q] T_j(u), stored as a double-float
// pair at the record's exponent of F.  Every thread of the block calls it (it holds
// block barriers); act selects the threads that own an (f, il, q), and the lanes of
// a warp that call it together span whole groups of Q (the shuffles run over a
// group); warps without such a thread (run false) only take the barriers.  With
// geometry, the record's mid and 1/half are written too.
template <int IPB>
__device__ __forceinline__ void series_fit(const Consts& c, const double (*sv)[IPB][kSeriesQ],
                                           double (*sf)[IPB][kSeriesQ], double (*sc)[IPB][kSeriesQ],
                                           const double (*dct)[kSeriesQ], const double (*tcoef)[kSeriesQ],
                                           int (*skf)[IPB], SeriesRec* __restrict__ tab, const int i, const bool run,
                                           const bool act, const int fa, const int il, const int q,
                                           const bool geometry, const double mid, const double half) {
    const int lane = threadIdx.x & 31;
    const int f = act ? fa : 0;  // (inactive threads read the first function and write nothing)
    if (run) {
        const double lz = sv[0][il][q], lg = sv[1][il][q];
        const double v = exp(f == 0 ? lz : f == 1 ? lg : fma(c.pG, lg, c.qZ * lz));
        if (act) sf[f][il][q] = v;
    }
    __syncthreads();
    if (run) {
        double acc = 0.0;
        for (int r = 0; r < kSeriesQ; ++r) acc = fma(sf[f][il][r], dct[q][r], acc);
        if (act) sc[f][il][q] = (q == 0 ? 1.0 : 2.0) / kSeriesQ * acc;
    }
    __syncthreads();
    SeriesRec& R = tab[i];
    if (run) {  // (warp-uniform: the shuffles below run over whole warps)
        double mono = 0.0;
        for (int j = q; j < kSeriesQ; ++j) mono = fma(sc[f][il][j], tcoef[j][q], mono);
        // the record's exponent of this function: the largest biased exponent of its
        // coefficients (the Q lanes of the interval)
        int E = (int)(((unsigned)__double2hiint(mono) >> 20) & 0x7ffu);
        for (int off = kSeriesQ / 2; off > 0; off >>= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, off));
        // double-float pair of mono 2^-(E - 1023): hi rounded to FP32, lo the rounded remainder
        const double ms = ldexp(mono, 1023 - E);
        const float hi = (float)ms;
        const float lo = (float)(ms - (double)hi);
        if (act) {
            // (Z and G interleaved: leading parts, then trailing parts)
            float* t = f < 2 ? &R.e[q].x + f : &R.w[q].x;
            t[0] = hi;
            t[f < 2 ? 2 : 1] = lo;
            if (q == 0) R.ex[f] = E;
        }
        // the degree from which on the polynomial's tail is summed in FP32 alone: the
        // smallest k >= 1 with sum_{k' >= k} |c_k'| <= 2^-30 |c_0| for all three
        // functions (c_0, the value at the interval's middle, is positive), so that
        // the FP32 rounding of the tail (16 roundings of 2^-24 at most) stays below
        // 2^-50 of the value
        double tail = fabs(ms);
        for (int off = 1; off < kSeriesQ; off <<= 1) {
            const double o = __shfl_down_sync(0xffffffffu, tail, off);
            if (q + off < kSeriesQ) tail += o;
        }
        const double c0 = __shfl_sync(0xffffffffu, ms, lane & ~(kSeriesQ - 1));
        int kq = (q >= 1 && tail <= 0x1p-30 * fabs(c0)) ? q : kSeriesQ;
        for (int off = kSeriesQ / 2; off > 0; off >>= 1) kq = min(kq, __shfl_xor_sync(0xffffffffu, kq, off));
        if (act && q == 0) skf[f][il] = kq;
    }
    __syncthreads();
    if (run && act && f == 0 && q == 0) {
        if (geometry) {
            R.mid = mid;
            R.invhalf = 1.0 / half;
        }
        R.ex[3] = max(skf[0][il], max(skf[1][il], skf[2][il]));
    }
}

// Two intervals per block of three warps (the batched build).  Warp f < 2 (0: ln Z,
// 1: ln G) evaluates its series by the compensated Clenshaw recurrence, lane
// (il, q) = (lane / Q, lane % Q) at the node s_q of interval 2 blk + il; meanwhile
// warp 2 builds the end-point record and the interpolation and monomial tables;
// then series_fit with thread (warp, il, q).
constexpr int kSeriesIntervalsPerBlock = 2;
constexpr int kSeriesThreads = 96;
static_assert(kSeriesIntervalsPerBlock * kSeriesQ == 32, "one warp holds one function of the block's intervals");

__device__ __forceinline__ void series_table_block(const Consts& c, const double* __restrict__ coef,
                                                   SeriesRec* __restrict__ tab, const int blk) {
    __shared__ double sv[2][kSeriesIntervalsPerBlock][kSeriesQ];  // ln Z, ln G
    __shared__ double sf[3][kSeriesIntervalsPerBlock][kSeriesQ];  // Z, G, W
    __shared__ double sc[3][kSeriesIntervalsPerBlock][kSeriesQ];
    __shared__ double tcoef[kSeriesQ][kSeriesQ];  // tcoef[j][k] = [u^k] T_j(u)
    __shared__ double dct[kSeriesQ][kSeriesQ];    // dct[k][r] = cos(pi k (r + 1/2)/Q)
    __shared__ double scf[2 * DSE_MAX_CHEB];      // a then b
    __shared__ int skf[3][kSeriesIntervalsPerBlock];  // FP32-tail degree per function
    __shared__ double smh[kSeriesIntervalsPerBlock][4];  // cos th0, cos th1, sin((th0 + th1)/2), sin(h/2)
    if (blk * kSeriesIntervalsPerBlock >= c.sM) return;  // (batched grids span the largest table)
    const int f = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int il = lane / kSeriesQ, q = lane % kSeriesQ;
    for (int j = threadIdx.x; j < c.n; j += blockDim.x) scf[j] = coef[j];
    if (f == 0 && lane < 4 * kSeriesIntervalsPerBlock) {
        // the geometry of series_interval, one sincos per lane
        const double h = kPi / c.sM;
        const int ii = blk * kSeriesIntervalsPerBlock + (lane >> 2), w = lane & 3;
        const double th0 = ii * h, th1 = (ii + 1) * h;
        const double x = w == 0 ? th0 : w == 1 ? th1 : w == 2 ? 0.5 * (th0 + th1) : 0.5 * h;
        double sn, cs;
        sincos(x, &sn, &cs);
        smh[lane >> 2][w] = w < 2 ? cs : sn;
    }
    const int i = blk * kSeriesIntervalsPerBlock + il;
    __syncthreads();  // coefficients and interval geometry staged
    const double mid = 0.5 * (smh[il][0] + smh[il][1]);
    const double half = smh[il][2] * smh[il][3];
    if (f < 2) {
        const DD sdd = series_node(mid, half, q);
        sv[f][il][q] = f == 0 ? series_comp(scf, c.NZ, sdd.hi, sdd.lo) : series_comp(scf + c.NZ, c.NG, sdd.hi, sdd.lo);
    } else {
        if (blk == 0 && lane < 4) series_endpoint(c, scf, lane, tab);
        for (int e = lane; e < kSeriesQ * kSeriesQ; e += 32) {
            const int k = e / kSeriesQ, r = e % kSeriesQ;
            dct[k][r] = cos(kPi * k * (r + 0.5) / kSeriesQ);
        }
        if (lane < kSeriesQ) series_tcoef_column(lane, tcoef);
    }
    __syncthreads();
    series_fit<kSeriesIntervalsPerBlock>(c, sv, sf, sc, dct, tcoef, skf, tab, i, true, true, f, il, q, true, mid,
                                         half);
}

__global__ void __launch_bounds__(kSeriesThreads) k_series_table_batched(const BatchProblem* __restrict__ P,
                                                              const double* __restrict__ coef_base) {
    const BatchProblem& B = P[blockIdx.y];
    if (!B.active || !B.stab) return;
    series_table_block(B.t.c, coef_base + B.coef_off, B.stab, blockIdx.x);
}

// The single-problem build.  The nodes depend on the table's geometry alone, so
// their Chebyshev values are formed once per plan (k_series_init): tq[(i Q + q) N + j]
// = T_j(s_q) of interval i as a double-double (T_0 entered as 1/2), by the
// recurrence T_{j+1} = 2 s T_j - T_{j-1} in double-double arithmetic (rounding
// ~2^-104 per step), together with the records' geometry and, in cst, the
// interpolation table dct[Q][Q] followed by the monomial table tcoef[Q][Q].  Per
// Newton matrix (k_series_table) the node values ln Z(s_q) = sum_j a_j T_j(s_q),
// ln G(s_q) = sum_j b_j T_j(s_q) are compensated dot products (Ogita, Rump and
// Oishi's Dot2: the exact product error by FMA, the exact sum error by TwoSum,
// both collected in FP64), each spread over four lanes whose partial results are
// combined by TwoSum: the series as computed in about twice the working
// precision, rounded once, like the compensated Clenshaw sums of the batched
// build.  One block of four warps per interval (32 dot products: 16 nodes x 2
// functions), so that the FP64 work of the build spreads over every SM.
constexpr int kSeriesDotThreads = 128;
constexpr int kSeriesDotLanes = 4;  // lanes per dot product
static_assert(kSeriesDotThreads == 2 * kSeriesQ * kSeriesDotLanes, "one thread per (function, node, part)");

__device__ __forceinline__ DD dd_mul(const DD a, const DD b) {
    const double p = a.hi * b.hi;
    double e = fma(a.hi, b.hi, -p);
    e = fma(a.hi, b.lo, e);
    e = fma(a.lo, b.hi, e);
    return dd_fast_two_sum(p, e);
}

__global__ void __launch_bounds__(64) k_series_init(const Consts c, double2* __restrict__ tq,
                                                    double* __restrict__ cst, SeriesRec* __restrict__ tab) {
    const int i = blockIdx.x;
    const int tid = threadIdx.x;
    if (tid < kSeriesQ) {
        double mid, half;
        series_interval(c.sM, i, mid, half);
        if (tid == 0) {
            tab[i].mid = mid;
            tab[i].invhalf = 1.0 / half;
        }
        const DD s = series_node(mid, half, tid);
        const DD s2 = {2.0 * s.hi, 2.0 * s.lo};
        double2* T = tq + ((size_t)i * kSeriesQ + tid) * c.N;
        DD tm = {1.0, 0.0}, tc = s;
        T[0] = make_double2(0.5, 0.0);
        if (c.N > 1) T[1] = make_double2(tc.hi, tc.lo);
        for (int j = 2; j < c.N; ++j) {
            const DD tn = dd_add(dd_mul(s2, tc), DD{-tm.hi, -tm.lo});
            T[j] = make_double2(tn.hi, tn.lo);
            tm = tc;
            tc = tn;
        }
    } else if (i == 0 && tid >= 32) {
        const int lane = tid - 32;
        for (int e = lane; e < kSeriesQ * kSeriesQ; e += 32) {
            const int k = e / kSeriesQ, r = e % kSeriesQ;
            cst[e] = cos(kPi * k * (r + 0.5) / kSeriesQ);
        }
        if (lane < kSeriesQ) series_tcoef_column(lane, reinterpret_cast<double(*)[kSeriesQ]>(cst + kSeriesQ * kSeriesQ));
    }
}

__global__ void __launch_bounds__(kSeriesDotThreads) k_series_table(const Consts c, const double* __restrict__ coef,
                                                                    const double2* __restrict__ tq,
                                                                    const double* __restrict__ cst,
                                                                    SeriesRec* __restrict__ tab) {
    __shared__ double sv[2][1][kSeriesQ];  // ln Z, ln G
    __shared__ double sf[3][1][kSeriesQ];  // Z, G, W
    __shared__ double sc[3][1][kSeriesQ];
    __shared__ double tcoef[kSeriesQ][kSeriesQ];
    __shared__ double dct[kSeriesQ][kSeriesQ];
    __shared__ int skf[3][1];
    const int i = blockIdx.x;
    const int tid = threadIdx.x;
    for (int e = tid; e < 2 * kSeriesQ * kSeriesQ; e += kSeriesDotThreads) {
        const double v = __ldg(&cst[e]);
        if (e < kSeriesQ * kSeriesQ) dct[e / kSeriesQ][e % kSeriesQ] = v;
        else tcoef[(e - kSeriesQ * kSeriesQ) / kSeriesQ][e % kSeriesQ] = v;
    }
    {
        const int chain = tid / kSeriesDotLanes, part = tid % kSeriesDotLanes;
        const int f = chain / kSeriesQ, q = chain % kSeriesQ;
        const int nf = f == 0 ? c.NZ : c.NG;
        const double* __restrict__ cf = coef + (f == 0 ? 0 : c.NZ);
        const double2* __restrict__ T = tq + ((size_t)i * kSeriesQ + q) * c.N;
        double s = 0.0, e = 0.0;
#pragma unroll 4
        for (int j = part; j < nf; j += kSeriesDotLanes) {
            const double2 t = __ldg(&T[j]);
            const double a = __ldg(&cf[j]);
            const double p = a * t.x;
            const double pe = fma(a, t.x, -p);
            const DD ts = dd_two_sum(s, p);
            e += ts.lo + fma(a, t.y, pe);
            s = ts.hi;
        }
        // the parts of a dot product (consecutive lanes): TwoSum of the leading sums,
        // the errors added (the same on every lane of the group)
#pragma unroll
        for (int off = 1; off < kSeriesDotLanes; off <<= 1) {
            const double so = __shfl_xor_sync(0xffffffffu, s, off);
            const double eo = __shfl_xor_sync(0xffffffffu, e, off);
            const DD ts = dd_two_sum(s, so);
            e = (e + eo) + ts.lo;
            s = ts.hi;
        }
        if (part == 0) sv[f][0][q] = s + e;
    }
    if (i == 0 && tid >= 64 && tid < 68) series_endpoint(c, coef, tid - 64, tab);
    __syncthreads();
    // threads 0 .. 3Q-1 (the first two warps) own (f, q) = (tid / Q, tid % Q); the
    // rest of the second warp runs along for its shuffles, the last two warps take
    // the barriers only
    series_fit<1>(c, sv, sf, sc, dct, tcoef, skf, tab, i, tid < 64, tid < 3 * kSeriesQ, tid / kSeriesQ, 0,
                  tid % kSeriesQ, false, 0.0, 0.0);
}

// ------------------------------------------------------------------------
// Per external momentum r (rows 0..Rc-1: collocation points, Rc: x_Z, Rc+1: x_G):
//   y-only contraction  Y_c[j] = sum_k U_c(r,k) phi_j(y_k),  c in {Q, M, G}
//   z-part              V_c[j] = sum over radial splits of Vpart
//   D[r] = (dPi_Z/da (NZ), dPi_Z/db (NG), dPi_G/da (NZ), dPi_G/db (NG), Pi_Z, Pi_G)
// with  dPi_Z/da_j = K/(3x) q (Y_Q + V_Q),  dPi_Z/db_j = K/(3x) (p (Y_Q + V_Q) + Y_M + V_M),
//       dPi_G/da_j = -K V_G,  dPi_G/db_j = -K Y_G   (Sec. 2 equations, derivative
// closure d ln G(u)/d b_j = d ln Z(u)/d a_j = phi_j(u)).
// For x_G = 0, z = y: the ghost row is y-only and V_G = Y_G.
constexpr int kRowBlock = 512;
constexpr int kRowJ = 32;                   // coefficients per block (one per lane)
constexpr int kRowKG = kRowBlock / kRowJ;   // radial-node groups per block
constexpr int kRowSplitsPer = (128 + kRowKG - 1) / kRowKG;  // splits per group held in registers (KS <= 128)
constexpr int kChunkK = 256;

// Grid: (row r, block of 32 coefficients).  Thread (k-group kg, lane) owns
// coefficient j = 32 jb + lane, the radial nodes kk = kg mod kRowKG of each chunk
// and the radial splits kg mod kRowKG; the kRowKG partial sums are combined in a
// fixed order at the end (sixteen groups: many L2 loads in flight per SM).
template <bool FULL>
__device__ __forceinline__ void rowreduce_block(const Consts& c, int Rt, int KS, int nch,
                                                const Rad* __restrict__ rad, const Ang* __restrict__ ang,
                                                const Row* __restrict__ rows, const YTab* __restrict__ ytab,
                                                const double* __restrict__ phiy, const double* __restrict__ Upart,
                                                const double* __restrict__ Vpart, double* __restrict__ D, const int r,
                                                const int jb) {
    __shared__ double sU[kChunkK][3];
    __shared__ float2 sUd[kChunkK][3];           // U at the chunk's scale, double-float
    __shared__ unsigned sEm[3][kRowBlock / 32];  // per-warp maxima of U's exponents
    __shared__ double sY[kRowKG][3][kRowJ];
    __shared__ double sV[kRowKG][3][kRowJ];
    __shared__ double sR[6][kRowJ];              // the six combined sums (Y_Q, Y_M, Y_G, V_Q, V_M, V_G)
    __shared__ double sS4;
    const int N = c.N;
    const int NZ = c.NZ, NG = c.NG, n = c.n, Rc = c.Rc;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int kg = tid >> 5;
    int rt;
    bool special = false;  // x_G = 0 ghost row
    if (r <= Rc) rt = r;
    else {
        if (c.x_G > 0.0) rt = Rc + 1;
        else { rt = -1; special = true; }
    }
    const int flags = special ? kRowGhost : rows[rt].flags;
    const bool gluon = (flags & kRowGluon) != 0;
    const bool ghost = (flags & kRowGhost) != 0;
    const bool do_pi = (jb == 0);
    // this row's radial tables (the split rule gives every row its own)
    rad += rad_offset(c, r);
    ytab += rad_offset(c, r);
    phiy += rad_offset(c, r) * N;
    if (special && kg == 0) {
        // sum_l w_l sin^4(theta_l) by warp 0 (fixed order)
        double s4 = 0.0;
        for (int l = lane; l < c.na; l += 32) s4 += ang[l].w * ang[l].s4;
        for (int off = 16; off > 0; off >>= 1) s4 += __shfl_xor_sync(kFullMask, s4, off);
        if (lane == 0) sS4 = s4;
    }
    const int j = jb * kRowJ + lane;
    double Y0 = 0.0, Y1 = 0.0, Y2 = 0.0;
    double P0 = 0.0, P1 = 0.0, P2 = 0.0;  // warp 0: sums of U for Pi
    __syncthreads();
    for (int kb = 0; kb < c.nr; kb += kChunkK) {
        const int kn = min(kChunkK, c.nr - kb);
        unsigned e0 = 0u, e1 = 0u, e2 = 0u;
        for (int kk = tid; kk < kn; kk += kRowBlock) {
            const int k = kb + kk;
            double u0 = 0.0, u1 = 0.0, u2 = 0.0;
            if (special) {
                const Rad rd = rad[k];
                const YTab yt = ytab[k];
                u2 = rd.W * yt.yG * yt.Z / (rd.y * rd.y) * sS4;
            } else {
                const double* up = Upart + ((size_t)rt * c.nr + k) * nch * 3;
                for (int ch = 0; ch < nch; ++ch) {
                    u0 += up[ch * 3 + 0];
                    u1 += up[ch * 3 + 1];
                    u2 += up[ch * 3 + 2];
                }
            }
            sU[kk][0] = u0;
            sU[kk][1] = u1;
            sU[kk][2] = u2;
            e0 = max(e0, ((unsigned)__double2hiint(u0) >> 20) & 0x7ffu);
            e1 = max(e1, ((unsigned)__double2hiint(u1) >> 20) & 0x7ffu);
            e2 = max(e2, ((unsigned)__double2hiint(u2) >> 20) & 0x7ffu);
        }
        // the chunk's scale per kind: the largest biased exponent of its U values
        if (FULL) {
            e0 = __reduce_max_sync(kFullMask, e0);
            e1 = __reduce_max_sync(kFullMask, e1);
            e2 = __reduce_max_sync(kFullMask, e2);
            if (lane == 0) {
                sEm[0][kg] = e0;
                sEm[1][kg] = e1;
                sEm[2][kg] = e2;
            }
        }
        __syncthreads();
        int E0 = 0, E1 = 0, E2 = 0;
        if (FULL) {
#pragma unroll
            for (int w = 0; w < kRowBlock / 32; ++w) {
                E0 = max(E0, (int)sEm[0][w]);
                E1 = max(E1, (int)sEm[1][w]);
                E2 = max(E2, (int)sEm[2][w]);
            }
            for (int kk = tid; kk < kn; kk += kRowBlock) {
                sUd[kk][0] = df_split(sU[kk][0], E0 - 1023);
                sUd[kk][1] = df_split(sU[kk][1], E1 - 1023);
                sUd[kk][2] = df_split(sU[kk][2], E2 - 1023);
            }
        }
        __syncthreads();
        if (do_pi && kg == 0) {
            for (int kk = lane; kk < kn; kk += 32) {
                P0 += sU[kk][0];
                P1 += sU[kk][1];
                P2 += sU[kk][2];
            }
        }
        if (FULL && j < N) {
            // the y-only contraction on the FP32 pipe: double-float products of the
            // scaled U and phi_j(y_k), renormalised every four nodes, widened once
            // per chunk (within ~2^-47 of the magnitudes it sums, like the z part)
            float2 a0 = make_float2(0.0f, 0.0f), a1 = a0, a2 = a0;
            int q = 0;
#pragma unroll 4
            for (int kk = kg; kk < kn; kk += kRowKG) {  // (unrolled: loads in flight, same order)
                const float2 ph = df_split(phiy[(size_t)(kb + kk) * N + j], 0);
                df_fma(a0, sUd[kk][0], ph);
                df_fma(a1, sUd[kk][1], ph);
                df_fma(a2, sUd[kk][2], ph);
                if ((++q & 3) == 0) {
                    df_renorm(a0);
                    df_renorm(a1);
                    df_renorm(a2);
                }
            }
            df_renorm(a0);
            df_renorm(a1);
            df_renorm(a2);
            Y0 += df_widen(a0.x, E0) + df_widen(a0.y, E0);
            Y1 += df_widen(a1.x, E1) + df_widen(a1.y, E1);
            Y2 += df_widen(a2.x, E2) + df_widen(a2.y, E2);
        }
        __syncthreads();
    }
    if (FULL) {
        sY[kg][0][lane] = Y0;
        sY[kg][1][lane] = Y1;
        sY[kg][2][lane] = Y2;
    }
    // the z-derivative sums of the radial splits kg, kg + kRowKG, ...: in
    // double-float at the thread's own scale (the largest exponent among its
    // values), widened once.  With KS <= 128 (every plan) the thread's values, at
    // most kRowSplitsPer per kind, are loaded once, all in flight, and scanned twice
    // in registers; more splits (large radial rules of a batch) take two passes over
    // memory.  Both add the same terms in the same order.
    if (FULL && !special && j < N) {
        const double* vp = Vpart + (size_t)rt * KS * 3 * N;
        unsigned m0 = 0u, m1 = 0u, m2 = 0u;
        float2 v0 = make_float2(0.0f, 0.0f), v1 = v0, v2 = v0;
        if (KS <= kRowSplitsPer * kRowKG) {
            double w0[kRowSplitsPer], w1[kRowSplitsPer], w2[kRowSplitsPer];
#pragma unroll
            for (int t = 0; t < kRowSplitsPer; ++t) {
                const int sp = kg + t * kRowKG;
                const bool in = sp < KS;
                w0[t] = in ? vp[(size_t)sp * 3 * N + j] : 0.0;
                w1[t] = in ? vp[(size_t)sp * 3 * N + N + j] : 0.0;
                w2[t] = in ? vp[(size_t)sp * 3 * N + 2 * N + j] : 0.0;
            }
#pragma unroll
            for (int t = 0; t < kRowSplitsPer; ++t) {
                m0 = max(m0, ((unsigned)__double2hiint(w0[t]) >> 20) & 0x7ffu);
                m1 = max(m1, ((unsigned)__double2hiint(w1[t]) >> 20) & 0x7ffu);
                m2 = max(m2, ((unsigned)__double2hiint(w2[t]) >> 20) & 0x7ffu);
            }
#pragma unroll
            for (int t = 0; t < kRowSplitsPer; ++t) {
                if (kg + t * kRowKG < KS) {
                    v0 = df_add(v0, df_split(w0[t], (int)m0 - 1023));
                    v1 = df_add(v1, df_split(w1[t], (int)m1 - 1023));
                    v2 = df_add(v2, df_split(w2[t], (int)m2 - 1023));
                }
            }
        } else {
#pragma unroll 4
            for (int sp = kg; sp < KS; sp += kRowKG) {
                m0 = max(m0, ((unsigned)__double2hiint(vp[(size_t)sp * 3 * N + j]) >> 20) & 0x7ffu);
                m1 = max(m1, ((unsigned)__double2hiint(vp[(size_t)sp * 3 * N + N + j]) >> 20) & 0x7ffu);
                m2 = max(m2, ((unsigned)__double2hiint(vp[(size_t)sp * 3 * N + 2 * N + j]) >> 20) & 0x7ffu);
            }
#pragma unroll 4
            for (int sp = kg; sp < KS; sp += kRowKG) {
                v0 = df_add(v0, df_split(vp[(size_t)sp * 3 * N + j], (int)m0 - 1023));
                v1 = df_add(v1, df_split(vp[(size_t)sp * 3 * N + N + j], (int)m1 - 1023));
                v2 = df_add(v2, df_split(vp[(size_t)sp * 3 * N + 2 * N + j], (int)m2 - 1023));
            }
        }
        sV[kg][0][lane] = df_widen(v0.x, (int)m0) + df_widen(v0.y, (int)m0);
        sV[kg][1][lane] = df_widen(v1.x, (int)m1) + df_widen(v1.y, (int)m1);
        sV[kg][2][lane] = df_widen(v2.x, (int)m2) + df_widen(v2.y, (int)m2);
    }
    __syncthreads();
    // the six sums over the groups in a fixed order, one per warp
    if (FULL && kg < 6 && j < N) {
        double v = 0.0;
        if (kg < 3) {
            for (int q = 0; q < kRowKG; ++q) v += sY[q][kg][lane];
        } else if (!special) {
            for (int q = 0; q < kRowKG; ++q) v += sV[q][kg - 3][lane];
        }
        sR[kg][lane] = v;
    }
    __syncthreads();
    const Row rw = rows[rt >= 0 ? rt : 0];
    const double pre = gluon ? rw.pre : 0.0;
    double* out = D + (size_t)r * ldD(c);
    if (FULL && kg == 0 && j < N) {
        const double y0 = sR[0][lane], y1 = sR[1][lane], y2 = sR[2][lane];
        const double VQ = sR[3][lane], VM = sR[4][lane];
        const double VG = special ? y2 : sR[5][lane];
        const double tq = y0 + VQ;
        if (j < NZ) {
            out[j] = gluon ? pre * c.qZ * tq : 0.0;
            out[n + j] = ghost ? -c.K * VG : 0.0;
        }
        if (j < NG) {
            out[NZ + j] = gluon ? pre * (c.pG * tq + y1 + VM) : 0.0;
            out[n + NZ + j] = ghost ? -c.K * y2 : 0.0;
        }
    }
    if (do_pi && kg == 0) {
        for (int off = 16; off > 0; off >>= 1) {
            P0 += __shfl_xor_sync(kFullMask, P0, off);
            P1 += __shfl_xor_sync(kFullMask, P1, off);
            P2 += __shfl_xor_sync(kFullMask, P2, off);
        }
        if (lane == 0) {
            out[2 * n] = gluon ? pre * (P0 + P1) : 0.0;
            out[2 * n + 1] = ghost ? -c.K * P2 : 0.0;
        }
    }
}

template <bool FULL>
__global__ void __launch_bounds__(kRowBlock) k_rowreduce(const Consts c, int Rt, int KS, int nch,
                                                         const Rad* __restrict__ rad, const Ang* __restrict__ ang,
                                                         const Row* __restrict__ rows, const YTab* __restrict__ ytab,
                                                         const double* __restrict__ phiy,
                                                         const double* __restrict__ Upart,
                                                         const double* __restrict__ Vpart, double* __restrict__ D) {
    rowreduce_block<FULL>(c, Rt, KS, nch, rad, ang, rows, ytab, phiy, Upart, Vpart, D, blockIdx.x, blockIdx.y);
}

// Grid (row, coefficient block, problem); rows and blocks past a problem's own
// counts return at once.
template <bool FULL>
__global__ void __launch_bounds__(kRowBlock) k_rowreduce_batched(const BatchProblem* __restrict__ P) {
    const BatchProblem& B = P[blockIdx.z];
    if (!B.active) return;
    const Consts& c = B.t.c;
    if ((int)blockIdx.x >= c.Rc + 2) return;
    if ((int)blockIdx.y >= (FULL ? (c.N + kRowJ - 1) / kRowJ : 1)) return;
    rowreduce_block<FULL>(c, B.t.Rt, B.t.KS, B.t.nch, B.t.rad, B.t.ang, B.t.rows, B.t.ytab, B.phiy, B.t.Upart,
                          B.t.Vpart, B.D, blockIdx.x, blockIdx.y);
}

// J and F from the per-row derivative vectors (Sec. 3 matrix layout; n = NZ + NG,
// gluon rows i < NZ at D row i, ghost rows i < NG at D row gofs + i):
//   J[i][j]      = -Z(x_i)^{-1} phi_j(x_i) [j < NZ] - dPi_Z(x_i)/dc_j + dPi_Z(x_Z)/dc_j
//   J[NZ+i][j]   = -G(x_i)^{-1} phi_{j-NZ}(x_i) [j >= NZ] - dPi_G(x_i)/dc_j + dPi_G(x_G)/dc_j
//   F[i]    = Z(x_i)^{-1} - Z(x_Z)^{-1} - Pi_Z(x_i) + Pi_Z(x_Z)
//   F[NZ+i] = G(x_i)^{-1} - G(x_G)^{-1} - Pi_G(x_i) + Pi_G(x_G)
// Entry (i, j) of J and entry i of F from the D vectors (the rows above).
__device__ __forceinline__ double assemble_J(const Consts& c, const XTab* __restrict__ xtab,
                                             const double* __restrict__ phix, const double* __restrict__ D,
                                             const int i, const int j) {
    const int N = c.N;
    const int NZ = c.NZ;
    const int n = c.n;
    const size_t ld = ldD(c);
    if (i < NZ) {
        const double* Di = D + (size_t)i * ld;
        const double* DZ = D + (size_t)c.Rc * ld;  // x_Z row
        if (j < NZ) return -xtab[i].Zinv * phix[(size_t)i * N + j] - Di[j] + DZ[j];
        return -Di[j] + DZ[j];
    }
    const int r = c.gofs + (i - NZ);
    const double* Di = D + (size_t)r * ld;
    const double* DG = D + (size_t)(c.Rc + 1) * ld;  // x_G row
    if (j < NZ) return -Di[n + j] + DG[n + j];
    return -xtab[r].Ginv * phix[(size_t)r * N + (j - NZ)] - Di[n + j] + DG[n + j];
}

__device__ __forceinline__ double assemble_F(const Consts& c, const XTab* __restrict__ xtab,
                                             const double* __restrict__ D, const int i) {
    const int n = c.n;
    const size_t ld = ldD(c);
    if (i < c.NZ) return xtab[i].Zinv - c.zinv_Z - D[(size_t)i * ld + 2 * n] + D[(size_t)c.Rc * ld + 2 * n];
    const int r = c.gofs + (i - c.NZ);
    return xtab[r].Ginv - c.ginv_G - D[(size_t)r * ld + 2 * n + 1] + D[(size_t)(c.Rc + 1) * ld + 2 * n + 1];
}

template <bool FULL>
__device__ __forceinline__ void assemble_range(const Consts& c, const XTab* __restrict__ xtab,
                                               const double* __restrict__ phix, const double* __restrict__ D,
                                               double* __restrict__ J, double* __restrict__ F,
                                               int* __restrict__ status, const size_t first, const size_t stride) {
    const int n = c.n;
    const size_t total = FULL ? (size_t)n * n : 0;
    bool bad = false;
    for (size_t e = first; e < total + n; e += stride) {
        if (e < total) {
            const double v = assemble_J(c, xtab, phix, D, (int)(e / n), (int)(e % n));
            J[e] = v;
            bad |= !isfinite(v);
        } else if (F) {
            const double v = assemble_F(c, xtab, D, (int)(e - total));
            F[e - total] = v;
            bad |= !isfinite(v);
        }
    }
    if (bad) atomicOr(status, kStatusNonfinite);
}

template <bool FULL>
__global__ void k_assemble(const Consts c, const XTab* __restrict__ xtab, const double* __restrict__ phix,
                           const double* __restrict__ D, double* __restrict__ J, double* __restrict__ F,
                           int* __restrict__ status) {
    assemble_range<FULL>(c, xtab, phix, D, J, F, status, blockIdx.x * (size_t)blockDim.x + threadIdx.x,
                         (size_t)gridDim.x * blockDim.x);
}

template <bool FULL>
__global__ void k_assemble_batched(const BatchProblem* __restrict__ P, double* __restrict__ J_base,
                                   double* __restrict__ F_base) {
    const BatchProblem& B = P[blockIdx.y];
    if (!B.active) return;
    double* J = J_base ? J_base + B.J_off : B.J;
    double* F = F_base ? F_base + B.coef_off : B.F;
    assemble_range<FULL>(B.t.c, B.xtab, B.phix, B.D, J, F, B.status, blockIdx.x * (size_t)blockDim.x + threadIdx.x,
                         (size_t)gridDim.x * blockDim.x);
}

// ------------------------------------------------------------------------
// Newton step (Sec. 3): J Delta = F by LU with partial pivoting (one block,
// matrix in place in global memory), then c <- c - rho Delta.  work holds
// 2n doubles (right-hand side, solution).  stats: ||F||_inf,
// ||diag(Z(x_i), G(x_i)) F||_inf, ||Delta||_inf.
constexpr int kLuThreads = 512;

__global__ void __launch_bounds__(kLuThreads) k_lu_newton(const Consts c, double* __restrict__ A,
                                                          const double* __restrict__ F,
                                                          const XTab* __restrict__ xtab, double* __restrict__ coef,
                                                          double rho, double* __restrict__ work,
                                                          double* __restrict__ stats, int* __restrict__ status,
                                                          const int* __restrict__ done) {
    // the FP32 LU path already took the step (dse_lu32.cu)
    if (done && *done) return;
    __shared__ double sv[kLuThreads / 32];
    __shared__ int si[kLuThreads / 32];
    __shared__ int s_piv;
    __shared__ int s_fail;
    __shared__ double s_red[3][kLuThreads / 32];
    const int n = c.n;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int WARPS = kLuThreads / 32;
    double* b = work;
    double* x = work + n;
    // norms of F (and a copy as right-hand side)
    double mF = 0.0, mS = 0.0;
    for (int i = tid; i < n; i += kLuThreads) {
        const double f = F[i];
        b[i] = f;
        const double sc = i < c.NZ ? xtab[i].Z : xtab[c.gofs + i - c.NZ].G;
        mF = fmax(mF, fabs(f));
        mS = fmax(mS, fabs(f) * sc);
        if (!isfinite(f)) mF = INFINITY;
    }
    for (int off = 16; off > 0; off >>= 1) {
        mF = fmax(mF, __shfl_xor_sync(kFullMask, mF, off));
        mS = fmax(mS, __shfl_xor_sync(kFullMask, mS, off));
    }
    if (lane == 0) {
        s_red[0][warp] = mF;
        s_red[1][warp] = mS;
    }
    if (tid == 0) s_fail = (*status) & (kStatusNonfinite | kStatusSingular);
    __syncthreads();
    if (tid == 0) {
        double a = 0.0, bb = 0.0;
        for (int w = 0; w < WARPS; ++w) {
            a = fmax(a, s_red[0][w]);
            bb = fmax(bb, s_red[1][w]);
        }
        stats[0] = a;
        stats[1] = bb;
        stats[2] = 0.0;
        stats[3] = -1.0;
        if (!isfinite(a)) s_fail |= kStatusNonfinite;
    }
    __syncthreads();
    if (s_fail) {
        if (tid == 0) atomicOr(status, s_fail);
        return;
    }
    for (int k = 0; k < n; ++k) {
        // pivot search in column k (ties: smallest row index)
        double best = -1.0;
        int bi = n;
        for (int i = k + tid; i < n; i += kLuThreads) {
            const double v = fabs(A[(size_t)i * n + k]);
            if (v > best || (v == best && i < bi)) {
                best = v;
                bi = i;
            }
        }
        for (int off = 16; off > 0; off >>= 1) {
            const double ov = __shfl_xor_sync(kFullMask, best, off);
            const int oi = __shfl_xor_sync(kFullMask, bi, off);
            if (ov > best || (ov == best && oi < bi)) {
                best = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            sv[warp] = best;
            si[warp] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            double bv = sv[0];
            int bix = si[0];
            for (int w = 1; w < WARPS; ++w)
                if (sv[w] > bv || (sv[w] == bv && si[w] < bix)) {
                    bv = sv[w];
                    bix = si[w];
                }
            s_piv = bix;
            if (!(bv > 1e-300) || !isfinite(bv)) s_fail = kStatusSingular;
        }
        __syncthreads();
        if (s_fail) break;
        const int p = s_piv;
        if (p != k) {
            for (int j = tid; j < n; j += kLuThreads) {
                const double t = A[(size_t)k * n + j];
                A[(size_t)k * n + j] = A[(size_t)p * n + j];
                A[(size_t)p * n + j] = t;
            }
            if (tid == 0) {
                const double t = b[k];
                b[k] = b[p];
                b[p] = t;
            }
        }
        __syncthreads();
        const double dkk = A[(size_t)k * n + k];
        for (int i = k + 1 + tid; i < n; i += kLuThreads) {
            const double l = A[(size_t)i * n + k] / dkk;
            A[(size_t)i * n + k] = l;
        }
        __syncthreads();
        const int m = n - k - 1;
        const double bk = b[k];
        for (int idx = tid; idx < m * m; idx += kLuThreads) {
            const int i = k + 1 + idx / m;
            const int j = k + 1 + idx % m;
            A[(size_t)i * n + j] = fma(-A[(size_t)i * n + k], A[(size_t)k * n + j], A[(size_t)i * n + j]);
        }
        for (int i = k + 1 + tid; i < n; i += kLuThreads) b[i] = fma(-A[(size_t)i * n + k], bk, b[i]);
        __syncthreads();
    }
    if (s_fail) {
        if (tid == 0) atomicOr(status, s_fail);
        return;
    }
    // back substitution
    for (int i = n - 1; i >= 0; --i) {
        if (tid == 0) x[i] = b[i] / A[(size_t)i * n + i];
        __syncthreads();
        const double xi = x[i];
        for (int t = tid; t < i; t += kLuThreads) b[t] = fma(-A[(size_t)t * n + i], xi, b[t]);
        __syncthreads();
    }
    double mD = 0.0;
    bool bad = false;
    for (int i = tid; i < n; i += kLuThreads) {
        mD = fmax(mD, fabs(x[i]));
        bad |= !isfinite(x[i]);
    }
    for (int off = 16; off > 0; off >>= 1) mD = fmax(mD, __shfl_xor_sync(kFullMask, mD, off));
    bad = __any_sync(kFullMask, bad);
    if (lane == 0) {
        s_red[2][warp] = mD;
        if (bad) atomicOr(&s_fail, kStatusNonfinite);
    }
    __syncthreads();
    if (tid == 0) {
        double a = 0.0;
        for (int w = 0; w < WARPS; ++w) a = fmax(a, s_red[2][w]);
        stats[2] = a;
    }
    if (s_fail) {
        if (tid == 0) atomicOr(status, s_fail);
        return;
    }
    for (int i = tid; i < n; i += kLuThreads) coef[i] = fma(-rho, x[i], coef[i]);
}

// ------------------------------------------------------------------------
// Newton step with an FP32 inverse and FP64 iterative refinement (for
// n = 2N <= kGjMaxN).  The FP64 rate is 1/64 of the FP32 rate on this GPU, so the
// O(n^3) part runs in FP32 and only O(n^2) work per refinement sweep runs in FP64:
//   1. rows of J scaled by exact powers of two (s_i = 2^-e_i, e_i = exponent of
//      max_j |J_ij|): A = diag(s) J, b = diag(s) F;
//   2. X ~ A^{-1} by Gauss-Jordan elimination with partial pivoting in FP32 on
//      [A | I] held in shared memory;
//   3. x <- x + X (b - A x) with the residual in FP64 until the correction is
//      below 2^-50 |x| (at most kRefineMax sweeps).
// If the sweeps do not converge (ill-conditioned J) the step falls back to the
// FP64 LU above in the same launch; the fallback also reports singular matrices.
constexpr int kGjThreads = 1024;
constexpr int kGjMaxN = 160;
constexpr int kRefineMax = 12;

__device__ void lu_fp64_block(int n, double* __restrict__ A, double* __restrict__ b, double* __restrict__ x,
                              int* s_fail, int* s_piv, double* sv, int* si) {
    const int tid = threadIdx.x;
    const int nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int warps = nt >> 5;
    for (int k = 0; k < n; ++k) {
        double best = -1.0;
        int bi = n;
        for (int i = k + tid; i < n; i += nt) {
            const double v = fabs(A[(size_t)i * n + k]);
            if (v > best || (v == best && i < bi)) {
                best = v;
                bi = i;
            }
        }
        for (int off = 16; off > 0; off >>= 1) {
            const double ov = __shfl_xor_sync(kFullMask, best, off);
            const int oi = __shfl_xor_sync(kFullMask, bi, off);
            if (ov > best || (ov == best && oi < bi)) {
                best = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            sv[warp] = best;
            si[warp] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            double bv = sv[0];
            int bix = si[0];
            for (int w = 1; w < warps; ++w)
                if (sv[w] > bv || (sv[w] == bv && si[w] < bix)) {
                    bv = sv[w];
                    bix = si[w];
                }
            *s_piv = bix;
            if (!(bv > 1e-300) || !isfinite(bv)) *s_fail = kStatusSingular;
        }
        __syncthreads();
        if (*s_fail) return;
        const int p = *s_piv;
        if (p != k) {
            for (int j = tid; j < n; j += nt) {
                const double t = A[(size_t)k * n + j];
                A[(size_t)k * n + j] = A[(size_t)p * n + j];
                A[(size_t)p * n + j] = t;
            }
            if (tid == 0) {
                const double t = b[k];
                b[k] = b[p];
                b[p] = t;
            }
        }
        __syncthreads();
        const double dkk = A[(size_t)k * n + k];
        for (int i = k + 1 + tid; i < n; i += nt) A[(size_t)i * n + k] /= dkk;
        __syncthreads();
        const int m = n - k - 1;
        const double bk = b[k];
        for (int idx = tid; idx < m * m; idx += nt) {
            const int i = k + 1 + idx / m;
            const int j = k + 1 + idx % m;
            A[(size_t)i * n + j] = fma(-A[(size_t)i * n + k], A[(size_t)k * n + j], A[(size_t)i * n + j]);
        }
        for (int i = k + 1 + tid; i < n; i += nt) b[i] = fma(-A[(size_t)i * n + k], bk, b[i]);
        __syncthreads();
    }
    for (int i = n - 1; i >= 0; --i) {
        if (tid == 0) x[i] = b[i] / A[(size_t)i * n + i];
        __syncthreads();
        const double xi = x[i];
        for (int t = tid; t < i; t += nt) b[t] = fma(-A[(size_t)t * n + i], xi, b[t]);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kGjThreads) k_newton_mixed(const Consts c, double* __restrict__ J,
                                                             const double* __restrict__ F,
                                                             const XTab* __restrict__ xtab,
                                                             double* __restrict__ coef, double rho,
                                                             double* __restrict__ work, double* __restrict__ stats,
                                                             int* __restrict__ status) {
    extern __shared__ __align__(16) float gj[];  // [n][2n]
    __shared__ double sv[kGjThreads / 32];
    __shared__ int si[kGjThreads / 32];
    __shared__ double s_x[2 * kGjMaxN];
    __shared__ double s_scale[2 * kGjMaxN];
    __shared__ float s_rf[2 * kGjMaxN];
    __shared__ int s_piv, s_fail, s_done;
    __shared__ float s_pinv;
    __shared__ double s_anorm;
    __shared__ double s_red[3][kGjThreads / 32];
    const int n = c.n;
    const int n2 = 2 * n;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int WARPS = kGjThreads / 32;

    // norms of F
    double mF = 0.0, mS = 0.0;
    for (int i = tid; i < n; i += kGjThreads) {
        const double f = F[i];
        const double sc = i < c.NZ ? xtab[i].Z : xtab[c.gofs + i - c.NZ].G;
        mF = fmax(mF, fabs(f));
        mS = fmax(mS, fabs(f) * sc);
        if (!isfinite(f)) mF = INFINITY;
    }
    for (int off = 16; off > 0; off >>= 1) {
        mF = fmax(mF, __shfl_xor_sync(kFullMask, mF, off));
        mS = fmax(mS, __shfl_xor_sync(kFullMask, mS, off));
    }
    if (lane == 0) {
        s_red[0][warp] = mF;
        s_red[1][warp] = mS;
    }
    if (tid == 0) {
        s_fail = (*status) & (kStatusNonfinite | kStatusSingular);
        s_done = 0;
    }
    __syncthreads();
    if (tid == 0) {
        double a = 0.0, bb = 0.0;
        for (int w = 0; w < WARPS; ++w) {
            a = fmax(a, s_red[0][w]);
            bb = fmax(bb, s_red[1][w]);
        }
        stats[0] = a;
        stats[1] = bb;
        stats[2] = 0.0;
        if (!isfinite(a)) s_fail |= kStatusNonfinite;
    }
    __syncthreads();
    if (s_fail) {
        if (tid == 0) atomicOr(status, s_fail);
        return;
    }

    // 1. exact power-of-two row scaling (one warp per row) and ||A||_inf
    double an = 0.0;
    for (int i = warp; i < n; i += WARPS) {
        double m = 0.0, rs = 0.0;
        for (int j = lane; j < n; j += 32) {
            const double v = fabs(J[(size_t)i * n + j]);
            m = fmax(m, v);
            rs += v;
        }
        for (int off = 16; off > 0; off >>= 1) {
            m = fmax(m, __shfl_xor_sync(kFullMask, m, off));
            rs += __shfl_xor_sync(kFullMask, rs, off);
        }
        if (lane == 0) {
            int e = 0;
            frexp(m, &e);
            const double sc = (m > 0.0 && isfinite(m)) ? ldexp(1.0, -e) : 0.0;
            s_scale[i] = sc;
            an = fmax(an, rs * sc);
        }
    }
    for (int off = 16; off > 0; off >>= 1) an = fmax(an, __shfl_xor_sync(kFullMask, an, off));
    if (lane == 0) s_red[2][warp] = an;
    __syncthreads();
    if (tid == 0) {
        double a = 0.0;
        for (int w = 0; w < WARPS; ++w) a = fmax(a, s_red[2][w]);
        s_anorm = a;
    }
    for (int i = tid; i < n; i += kGjThreads)
        if (s_scale[i] == 0.0) s_fail = kStatusSingular;  // benign race: same value
    __syncthreads();
    // 2. FP32 Gauss-Jordan on [A | I]
    if (!s_fail) {
        for (int i = warp; i < n; i += WARPS) {
            const double sc = s_scale[i];
            for (int j = lane; j < n2; j += 32)
                gj[i * n2 + j] = j < n ? (float)(J[(size_t)i * n + j] * sc) : ((j - n == i) ? 1.0f : 0.0f);
        }
        __syncthreads();
        for (int k = 0; k < n; ++k) {
            float best = -1.0f;
            int bi = n;
            for (int i = k + tid; i < n; i += kGjThreads) {
                const float v = fabsf(gj[i * n2 + k]);
                if (v > best || (v == best && i < bi)) {
                    best = v;
                    bi = i;
                }
            }
            for (int off = 16; off > 0; off >>= 1) {
                const float ov = __shfl_xor_sync(kFullMask, best, off);
                const int oi = __shfl_xor_sync(kFullMask, bi, off);
                if (ov > best || (ov == best && oi < bi)) {
                    best = ov;
                    bi = oi;
                }
            }
            if (lane == 0) {
                sv[warp] = best;
                si[warp] = bi;
            }
            __syncthreads();
            if (tid == 0) {
                double bv = sv[0];
                int bix = si[0];
                for (int w = 1; w < WARPS; ++w)
                    if (sv[w] > bv || (sv[w] == bv && si[w] < bix)) {
                        bv = sv[w];
                        bix = si[w];
                    }
                s_piv = bix;
                if (!(bv > 1e-30)) s_done = -1;  // numerically singular in FP32: use the FP64 path
                else s_pinv = 1.0f / gj[bix * n2 + k];
            }
            __syncthreads();
            if (s_done < 0) break;
            const int p = s_piv;
            // swap rows k and p, then scale row k by 1/pivot
            const float inv = s_pinv;
            for (int j = tid; j < n2; j += kGjThreads) {
                const float a = gj[k * n2 + j];
                const float bq = gj[p * n2 + j];
                gj[k * n2 + j] = bq * inv;
                if (p != k) gj[p * n2 + j] = a;
            }
            __syncthreads();
            // eliminate column k from every other row (one warp per row)
            for (int i = warp; i < n; i += WARPS) {
                if (i == k) continue;
                const float f = gj[i * n2 + k];
                for (int j = lane; j < n2; j += 32)
                    if (j != k) gj[i * n2 + j] = fmaf(-f, gj[k * n2 + j], gj[i * n2 + j]);
            }
            __syncthreads();
            for (int i = tid; i < n; i += kGjThreads)
                if (i != k) gj[i * n2 + k] = 0.0f;
            __syncthreads();
        }
    }
    // 3. refinement sweeps: x <- x + X (b - A x), residual in FP64, until the
    //    scaled residual is at the FP64 level of a backward-stable solve:
    //    max|r| <= 4 sqrt(n) 2^-53 ||A||_inf ||x||_inf
    bool converged = false;
    int sweeps = 0;
    if (!s_fail && s_done == 0) {
        for (int i = tid; i < n; i += kGjThreads) s_x[i] = 0.0;
        __syncthreads();
        const double tolfac = 4.0 * sqrt((double)n) * 0x1p-53 * s_anorm;
        for (int it = 0; it <= kRefineMax; ++it) {
            double rm = 0.0, xm = 0.0;
            for (int i = warp; i < n; i += WARPS) {
                double acc = 0.0;
                for (int j = lane; j < n; j += 32) acc = fma(J[(size_t)i * n + j], s_x[j], acc);
                for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(kFullMask, acc, off);
                if (lane == 0) {
                    const double r = s_scale[i] * (F[i] - acc);
                    s_rf[i] = (float)r;
                    rm = fmax(rm, fabs(r));
                    xm = fmax(xm, fabs(s_x[i]));
                    if (!isfinite(r)) rm = INFINITY;
                }
            }
            for (int off = 16; off > 0; off >>= 1) {
                rm = fmax(rm, __shfl_xor_sync(kFullMask, rm, off));
                xm = fmax(xm, __shfl_xor_sync(kFullMask, xm, off));
            }
            if (lane == 0) {
                s_red[0][warp] = rm;
                s_red[1][warp] = xm;
            }
            __syncthreads();
            double RM = 0.0, XM = 0.0;
            for (int w = 0; w < WARPS; ++w) {
                RM = fmax(RM, s_red[0][w]);
                XM = fmax(XM, s_red[1][w]);
            }
            if (!isfinite(RM)) break;
            if (RM <= tolfac * XM) {
                converged = true;
                break;
            }
            if (it == kRefineMax) break;
            ++sweeps;
            for (int i = warp; i < n; i += WARPS) {
                float acc = 0.0f;
                for (int j = lane; j < n; j += 32) acc = fmaf(gj[i * n2 + n + j], s_rf[j], acc);
                for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(kFullMask, acc, off);
                if (lane == 0) s_x[i] += (double)acc;
            }
            __syncthreads();
        }
    }
    double* xres = work + n;
    if (!s_fail && converged) {
        for (int i = tid; i < n; i += kGjThreads) xres[i] = s_x[i];
        __syncthreads();
    } else if (!s_fail) {
        // FP64 LU fallback on J (in place), right-hand side copied to work
        for (int i = tid; i < n; i += kGjThreads) work[i] = F[i];
        __syncthreads();
        lu_fp64_block(n, J, work, xres, &s_fail, &s_piv, sv, si);
        __syncthreads();
    }
    if (s_fail) {
        if (tid == 0) atomicOr(status, s_fail);
        return;
    }
    double mD = 0.0;
    bool bad = false;
    for (int i = tid; i < n; i += kGjThreads) {
        mD = fmax(mD, fabs(xres[i]));
        bad |= !isfinite(xres[i]);
    }
    for (int off = 16; off > 0; off >>= 1) mD = fmax(mD, __shfl_xor_sync(kFullMask, mD, off));
    bad = __any_sync(kFullMask, bad);
    if (lane == 0) {
        s_red[2][warp] = mD;
        if (bad) atomicOr(&s_fail, kStatusNonfinite);
    }
    __syncthreads();
    if (tid == 0) {
        double a = 0.0;
        for (int w = 0; w < WARPS; ++w) a = fmax(a, s_red[2][w]);
        stats[2] = a;
        stats[3] = converged ? (double)sweeps : -1.0;
    }
    if (s_fail) {
        if (tid == 0) atomicOr(status, s_fail);
        return;
    }
    for (int i = tid; i < n; i += kGjThreads) coef[i] = fma(-rho, xres[i], coef[i]);
}

// ------------------------------------------------------------------------
// Row scaling for the Newton step (one block per row of J, many SMs): the
// exact power of two s_i = 2^(1022 - E_i), E_i the largest biased exponent in
// row i (integer arithmetic on the exponent fields), A_i = s_i J_i converted to
// FP32, and the row sum of |A_i| (for ||A||_inf).  A zero row is singular.
constexpr int kScaleThreads = 128;
constexpr int kColPad = 144;  // >= 128 + 16 - 1, multiple of 4
constexpr int kGjBlock = 4;   // pivots per round of the blocked elimination
constexpr int kGjCols = 4;    // columns per lane of the panel warp (n <= 128)
static_assert(kGjCols * 32 <= 128, "the pivot keys hold the column in 7 bits");

__device__ __forceinline__ void scale_row(int n, const double* __restrict__ J, float* __restrict__ As,
                                          double2* __restrict__ rowinfo, int* __restrict__ status, const int i) {
    __shared__ int s_e[kScaleThreads / 32];
    __shared__ float s_sum[kScaleThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double* row = J + (size_t)i * n;
    int e = 0;
    for (int j = tid; j < n; j += kScaleThreads) e = max(e, (__double2hiint(row[j]) >> 20) & 0x7ff);
    e = __reduce_max_sync(kFullMask, e);
    if (lane == 0) s_e[warp] = e;
    __syncthreads();
    int E = s_e[0];
    for (int w = 1; w < kScaleThreads / 32; ++w) E = max(E, s_e[w]);
    // E = 0: zero (or subnormal) row; E = 0x7ff: Inf/NaN (already flagged by the assembly)
    const bool ok = E > 0 && E < 0x7ff;
    const double sc = ok ? __hiloint2double((1022 - E + 1023) << 20, 0) : 0.0;
    float sum = 0.0f;
    for (int j = tid; j < n; j += kScaleThreads) {
        const float a = ok ? (float)(row[j] * sc) : 0.0f;
        As[(size_t)i * n + j] = a;
        sum += fabsf(a);
    }
    for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(kFullMask, sum, off);
    if (lane == 0) s_sum[warp] = sum;
    __syncthreads();
    if (tid == 0) {
        float t = 0.0f;
        for (int w = 0; w < kScaleThreads / 32; ++w) t += s_sum[w];
        rowinfo[i] = make_double2(sc, (double)t);
        if (!ok) atomicOr(status, E == 0 ? kStatusSingular : kStatusNonfinite);
    }
}

__global__ void __launch_bounds__(kScaleThreads) k_scale_rows(int n, const double* __restrict__ J,
                                                              float* __restrict__ As, double2* __restrict__ rowinfo,
                                                              int* __restrict__ status) {
    scale_row(n, J, As, rowinfo, status, blockIdx.x);
}

// The assembly of row i of J (and of F[i]) followed by its scaling, one block
// per row: the same entries as k_assemble and the same scaled row as
// k_scale_rows (which re-reads the row this block has just written), in one
// launch instead of two dependent ones.
__global__ void __launch_bounds__(kScaleThreads)
    k_assemble_scale(const Consts c, const XTab* __restrict__ xtab, const double* __restrict__ phix,
                     const double* __restrict__ D, double* __restrict__ J, double* __restrict__ F,
                     float* __restrict__ As, double2* __restrict__ rowinfo, int* __restrict__ status) {
    const int n = c.n;
    const int i = blockIdx.x;
    bool bad = false;
    for (int j = threadIdx.x; j < n; j += kScaleThreads) {
        const double v = assemble_J(c, xtab, phix, D, i, j);
        J[(size_t)i * n + j] = v;
        bad |= !isfinite(v);
    }
    if (F && threadIdx.x == 0) {
        const double v = assemble_F(c, xtab, D, i);
        F[i] = v;
        bad |= !isfinite(v);
    }
    if (bad) atomicOr(status, kStatusNonfinite);
    __syncthreads();  // the row's stores are visible to the whole block
    scale_row(n, J, As, rowinfo, status, i);
}

__global__ void __launch_bounds__(kScaleThreads) k_scale_rows_batched(const BatchProblem* __restrict__ P) {
    const BatchProblem& B = P[blockIdx.y];
    if (!B.active || (int)blockIdx.x >= B.t.c.n) return;
    scale_row(B.t.c.n, B.J, B.As, B.rowinfo, B.status, blockIdx.x);
}

// FP64 iterative refinement for J x = F with an approximate inverse X of the
// row-scaled matrix diag(Sc) J: x <- x + X (Sc (F - J x)), with the residual in FP64
// (J in shared memory, one thread per row; F itself for the starting x = 0) and the
// products X r in FP32, until max |Sn (F - J x)| <= tolfac max |x| (a
// backward-stable solution for the row scaling Sn).  Returns 1 (converged) or 2
// (gave up: not finite or maxit sweeps; with early_abort also when a sweep reduces
// the residual by less than kReuseRate or the observed rate predicts more than
// maxit sweeps in all).  Called by every thread of the block; s_x holds x (zero
// on entry).  A sweep costs one FP64 matrix-vector product on this SM (~4 us at
// n = 128) against ~190 us for an elimination, so a kept inverse that contracts
// by 0.1 per sweep still pays.
constexpr int kReuseMax = 24;
constexpr double kReuseRate = 0.5;

// Row stride of the FP64 copy of J in shared memory: at least n and 4 mod 16
// doubles, so that the loads of the residual (four threads per row, columns
// j = part + 4 t, eight rows per warp) fall two by two into distinct bank pairs.
__host__ __device__ inline int reg_ldj(int n) { return (n + 11) / 16 * 16 + 4; }

// Upper bound of a non-negative double as a 32-bit key that orders like it (its
// high word, plus one unit unless the low word is zero), and the double of a key
// (which the key bounds from above when it came from key_up).
__device__ __forceinline__ unsigned key_up(double v) {
    const unsigned hi = (unsigned)__double2hiint(v);
    return hi + (__double2loint(v) != 0 && hi < 0x7ff00000u ? 1u : 0u);
}
__device__ __forceinline__ double key_value(unsigned k) { return __hiloint2double((int)k, 0); }

// ---- the residual over a thread-block cluster ----
// With n > 64 the Newton-step kernel runs as a cluster of ceil(n / 16) CTAs: CTA 0
// does the elimination and the refinement; every CTA (CTA 0 included) holds 16
// rows of J and forms their part of each refinement sweep's FP64 residual, so that
// the n^2 FP64 FMAs of a sweep, which on one SM take ~4.7 us at n = 128 (the FP64
// rate of one SM), spread over up to eight SMs.  CTA 0 writes x, the round's
// command and the row scales into the other CTAs' shared memory, and they write
// their rows of S r and their maxima keys into CTA 0's (distributed shared memory).
// A sweep is one round of two cluster barriers: (1) CTA 0 has written x and the
// command, (2) every CTA has written its rows.  CTA 0 ends with a stop command and
// one more round, so every CTA passes the same number of cluster barriers.
__shared__ int s_ncmd[2];  // 0 stop, 1 residual, 2 residual at x = 0; Sc is the kept scale

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_ctas() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
// every thread of every CTA of the cluster: the writes before it are visible after it
// (called where every thread of the block arrives; the warp is reconverged first,
// as the aligned forms require)
__device__ __forceinline__ void cluster_barrier() {
    __syncwarp();
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// the address of this CTA's shared variable p in CTA rank of the cluster
__device__ __forceinline__ unsigned cluster_addr(const void* p, unsigned rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"((unsigned)__cvta_generic_to_shared(p)), "r"(rank));
    return r;
}
__device__ __forceinline__ void cluster_st_f32(unsigned a, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void cluster_st_u32(unsigned a, unsigned v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void cluster_st_f64(unsigned a, double v) {
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}
__device__ __forceinline__ void cluster_st_s32(unsigned a, int v) {
    asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// (J x)[row] for one of a CTA's 16 rows: eight threads per row (threads 0 .. 127,
// part = tid mod 8) over the columns j = part + 8 t in two chains, combined over
// the eight by shuffles (every lane of warps 0 .. 3 takes part; dot = false: 0)
__device__ __forceinline__ double cl_row_dot(const double* __restrict__ Jr, const double* __restrict__ x, int n,
                                             int part, bool dot) {
    double a0 = 0.0, a1 = 0.0;
    if (dot) {
        int jj = part;
#pragma unroll 2
        for (; jj + 8 < n; jj += 16) {
            a0 = fma(Jr[jj], x[jj], a0);
            a1 = fma(Jr[jj + 8], x[jj + 8], a1);
        }
        if (jj < n) a0 = fma(Jr[jj], x[jj], a0);
    }
    double acc = a0 + a1;
    acc += __shfl_xor_sync(kFullMask, acc, 1);
    acc += __shfl_xor_sync(kFullMask, acc, 2);
    acc += __shfl_xor_sync(kFullMask, acc, 4);
    return acc;
}

// CTAs 1 .. of the cluster: rows 16 rank .. 16 rank + 15 of every sweep's residual
// until CTA 0 sends the stop command.  Jl: this CTA's dynamic shared memory; s_x,
// s_scale, s_sold hold what CTA 0 wrote (x, the row scales Sn and the kept ones);
// s_rf, s_red are this CTA's copies of CTA 0's variables (the same offsets in every
// CTA of the kernel), mapped to CTA 0's.
__device__ __noinline__ void newton_residual_rows(int n, int ldj, const double* __restrict__ J,
                                                  const double* __restrict__ F, double* Jl, const double* s_x,
                                                  const double* s_scale, const double* s_sold, const float* s_rf,
                                                  const unsigned* s_red, unsigned rank) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r0 = 16 * (int)rank;
    for (int rr = warp; rr < 16; rr += kGjThreads / 32) {
        const int i = r0 + rr;
        for (int jj = lane; jj < n; jj += 32) Jl[rr * ldj + jj] = i < n ? J[(size_t)i * n + jj] : 0.0;
    }
    const int row = r0 + (tid >> 3), part = tid & 7;
    const bool head = tid < 128 && part == 0 && row < n;  // the thread that finishes its row
    const double Fr = head ? F[row] : 0.0;
    const unsigned a_rf = cluster_addr(s_rf, 0), a_red = cluster_addr(s_red, 0);
    __syncthreads();
    for (;;) {
        cluster_barrier();  // (1)
        const int cmd = s_ncmd[0];
        if (cmd == 0) break;
        const int sel = s_ncmd[1];
        const double sn = head ? s_scale[row] : 0.0;
        const double sc = head ? (sel ? s_sold[row] : sn) : 0.0;
        if (tid < 128) {
            const double acc = cl_row_dot(Jl + (tid >> 3) * ldj, s_x, n, part, cmd == 1 && row < n);
            unsigned rk = 0u, xk = 0u;
            if (head) {
                const double r = Fr - acc;
                cluster_st_f32(a_rf + 4u * (unsigned)row, (float)(sc * r));
                const double rn = sn * r;
                rk = isfinite(rn) ? key_up(fabs(rn)) : 0x7ff00000u;
                xk = cmd == 1 ? (unsigned)__double2hiint(fabs(s_x[row])) : 0u;
            }
            rk = __reduce_max_sync(kFullMask, rk);
            xk = __reduce_max_sync(kFullMask, xk);
            if (lane == 0) {
                const unsigned slot = 4u * rank + (unsigned)warp;
                cluster_st_u32(a_red + 4u * slot, rk);
                cluster_st_u32(a_red + 4u * (32u + slot), xk);
            }
        }
        cluster_barrier();  // (2)
    }
    cluster_barrier();  // (2) of the stop round
}

__device__ __forceinline__ int refine_fp64(int n, int ldj, const double* Js, const float* Xs, const double* Sc,
                                           const double* Sn, const double* __restrict__ F, double* s_x, float* s_rf,
                                           unsigned (*s_red)[32], int* s_conv, double tolfac, int maxit,
                                           bool early_abort, int* sweeps, const bool cl) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double prev = INFINITY;  // lane 0 of warp 0 only
    int st = 0;
    const int ncta = cl ? (int)cluster_ctas() : 1;
    for (int it = 0; it <= maxit; ++it) {
        if (cl) {
            // in a cluster: the command into every other CTA, at the first round the
            // row scales of its rows (x reached them with the last update; x = 0 at
            // the first round), then this CTA's rows 0 .. 15 (the others' meanwhile)
            if (tid >= 1 && tid < ncta) {
                cluster_st_s32(cluster_addr(&s_ncmd[0], (unsigned)tid), it > 0 ? 1 : 2);
                cluster_st_s32(cluster_addr(&s_ncmd[1], (unsigned)tid), Sc != Sn ? 1 : 0);
            }
            if (it == 0 && tid >= 16 && tid < n && (tid >> 4) < ncta) {
                const unsigned h = (unsigned)tid >> 4;  // the CTA that holds row tid
                cluster_st_f64(cluster_addr(Sn + tid, h), Sn[tid]);
                if (Sc != Sn) cluster_st_f64(cluster_addr(Sc + tid, h), Sc[tid]);
            }
            cluster_barrier();  // (1) x and the command
            if (tid < 128) {
                const int row = tid >> 3, part = tid & 7;
                const double acc = cl_row_dot(Js + row * ldj, s_x, n, part, it > 0 && row < n);
                unsigned rk = 0u, xk = 0u;
                if (part == 0 && row < n) {
                    const double r = F[row] - acc;
                    s_rf[row] = (float)(Sc[row] * r);
                    const double rn = Sn[row] * r;
                    rk = isfinite(rn) ? key_up(fabs(rn)) : 0x7ff00000u;
                    xk = (unsigned)__double2hiint(fabs(s_x[row]));
                }
                rk = __reduce_max_sync(kFullMask, rk);
                xk = __reduce_max_sync(kFullMask, xk);
                if (lane == 0) {
                    s_red[0][warp] = rk;
                    s_red[1][warp] = xk;
                }
            }
            cluster_barrier();  // (2) every CTA's rows of S r and its keys
        } else if (tid < 512) {
        // residual: four threads per row (16 warps), each over the columns
        // j = part + 4 t in two chains; the maxima of |S r| and |x| as integer keys
        // (one warp reduction each; the residual's key rounded up, x's down)
            unsigned rk = 0u, xk = 0u;
            const int row = tid >> 2, part = tid & 3;
            double acc = 0.0;
            if (row < n && it > 0) {  // x = 0 at the start: r = F
                const double* Jr = Js + (size_t)row * ldj;
                double a0 = 0.0, a1 = 0.0;
                int jj = part;
#pragma unroll 4
                for (; jj + 4 < n; jj += 8) {
                    a0 = fma(Jr[jj], s_x[jj], a0);
                    a1 = fma(Jr[jj + 4], s_x[jj + 4], a1);
                }
                if (jj < n) a0 = fma(Jr[jj], s_x[jj], a0);
                acc = a0 + a1;
            }
            acc += __shfl_xor_sync(kFullMask, acc, 1);
            acc += __shfl_xor_sync(kFullMask, acc, 2);
            if (row < n && part == 0) {
                const double r = F[row] - acc;
                s_rf[row] = (float)(Sc[row] * r);
                const double rn = Sn[row] * r;
                rk = isfinite(rn) ? key_up(fabs(rn)) : 0x7ff00000u;
                xk = (unsigned)__double2hiint(fabs(s_x[row]));
            }
            rk = __reduce_max_sync(kFullMask, rk);
            xk = __reduce_max_sync(kFullMask, xk);
            if (lane == 0) {
                s_red[0][warp] = rk;
                s_red[1][warp] = xk;
            }
        }
        __syncthreads();
        if (warp == 0) {
            // the maxima over the 32 slots (16 warps here, or 4 per CTA of a
            // cluster; unused slots hold 0), the decision by lane 0
            const unsigned RK = __reduce_max_sync(kFullMask, s_red[0][lane]);
            const unsigned XK = __reduce_max_sync(kFullMask, s_red[1][lane]);
            if (lane == 0) {
                const double RM = key_value(RK), XM = key_value(XK);
                int v = 0;  // 0: continue, 1: converged, 2: give up
                if (!(RK < 0x7ff00000u)) v = 2;
                else if (RM <= tolfac * XM) v = 1;
                else if (it == maxit) v = 2;
                else if (early_abort && it > 0) {
                    // observed contraction; sweeps still needed at that rate (FP32
                    // logarithms: an estimate of a count)
                    const float rate = (float)(RM / prev);
                    if (!(rate <= (float)kReuseRate)) v = 2;
                    else if ((float)it + __log2f((float)(tolfac * XM / RM)) / __log2f(rate) > (float)maxit) v = 2;
                }
                prev = RM;
                *s_conv = v;
            }
        }
        __syncthreads();
        st = *s_conv;
        if (st) break;
        ++*sweeps;
        // x += X r  (FP32 products, 8 threads per row; the four rows of a warp start
        // at columns 8 apart, so that their shared-memory reads use distinct banks)
        {
            const int i = tid >> 3, part = tid & 7;
            const int n8 = (n + 7) & ~7;
            const int rot = 8 * (i & 3);
            float acc = 0.0f;
            if (i < n) {
#pragma unroll 4
                for (int t = part; t < n8; t += 8) {
                    int jj = t + rot;
                    if (jj >= n8) jj -= n8;
                    if (jj < n) acc = fmaf(Xs[i * n + jj], s_rf[jj], acc);
                }
            }
            acc += __shfl_xor_sync(kFullMask, acc, 4);
            acc += __shfl_xor_sync(kFullMask, acc, 2);
            acc += __shfl_xor_sync(kFullMask, acc, 1);
            if (part == 0 && i < n) {
                const double xn = s_x[i] + (double)acc;
                s_x[i] = xn;
                // (in a cluster, x of the next sweep into every other CTA)
                for (int h = 1; h < ncta; ++h) cluster_st_f64(cluster_addr(s_x + i, (unsigned)h), xn);
            }
        }
        __syncthreads();
    }
    return st;
}

// ------------------------------------------------------------------------
// Newton step for n = NZ + NG <= 128 on one SM, FP64 work kept to O(n^2):
//   - the row-scaled FP32 matrix A = diag(s) J (k_scale_rows) is inverted in
//     place by Gauss-Jordan elimination held in registers: thread t owns column
//     j = t mod n of the R consecutive rows g R .. g R + R - 1 (g = t div n);
//   - pivoting is by columns (partial pivoting of A^T): step k takes the
//     largest unused entry of row k, so the row of the step is static and the
//     loop over it unrolls with every register index known at compile time;
//     row k and the pivot column travel through double-buffered shared memory,
//     two barriers per step, R FMAs per thread;
//   - with pivot column q_k at step k the inverse is X[q_k][m] = a[k][q_m];
//   - x <- x + X (b - A x) with the residual in FP64 (J copied to shared
//     memory, one thread per row) until max|r| <= 4 sqrt(n) 2^-53 ||A|| ||x||;
//   - with Xg given, the inverse that solved the previous Newton step (and its
//     row scales) is kept in global memory and tried first: late Newton steps
//     change J little, so refinement sweeps with the old X reach the same
//     backward error and the elimination is skipped; if the observed contraction
//     per sweep is above kReuseRate, or predicts more than kReuseMax sweeps in
//     all, the step eliminates afresh; after a failed attempt the next one waits
//     for an update ten times smaller than the one that preceded the failure;
//   - FP64 LU fallback if the sweeps stall.
// One warp pivots the panel of a round in registers (lane L holds columns L + 32 c):
// rows k0 .. k0 + nb - 1 of the partly eliminated matrix, with column pivoting.
// Writes the final panel rows back, the pivot columns to s_q[k0 ..], the columns
// used so far to s_used, and *s_done = -1 on a pivot below 1e-30.  Not inlined: the
// pivot chain gets the registers that the caller's rows hold meanwhile.
__device__ __noinline__ void gj_pivot_panel(float (*panel)[128], const int k0, const int nb, const int n,
                                            const int lane, unsigned char* s_used, int* s_q, int* s_done) {
        float P[kGjBlock][kGjCols];
        bool ucol[kGjCols];
#pragma unroll
        for (int cc = 0; cc < kGjCols; ++cc) {
            const int col = lane + 32 * cc;
            ucol[cc] = col >= n || s_used[col] != 0;
#pragma unroll
            for (int p = 0; p < kGjBlock; ++p) P[p][cc] = (col < n && p < nb) ? panel[p][col] : 0.0f;
        }
        bool sing = false;
#pragma unroll
        for (int p = 0; p < kGjBlock; ++p) {
            if (p < nb && !sing) {  // uniform over the warp
                // pivot column: the largest unused entry of panel row p,
                // by one warp reduction over keys that hold |a| as bits
                // (monotonic for non-negative floats) cut to 16 fraction
                // bits, and 127 - column in the 7 bits below: of entries
                // equal to 2^-16 the lowest column wins (pivoted columns: 0)
                unsigned key = 0u;
#pragma unroll
                for (int cc = 0; cc < kGjCols; ++cc) {
                    const unsigned ab = (unsigned)__float_as_int(fabsf(P[p][cc])) & 0xffffff80u;
                    const unsigned bv = ucol[cc] ? 0u : (ab | (unsigned)(127 - (lane + 32 * cc)));
                    key = max(key, bv);
                }
                const unsigned mk = __reduce_max_sync(kFullMask, key);
                const int idx = 127 - (int)(mk & 0x7fu);
                const float a = __int_as_float((int)(mk & 0xffffff80u));
                if (!(a > 1e-30f)) {
                    if (lane == 0) *s_done = -1;
                    sing = true;
                } else {
                    const int q = idx;
                    const int ql = q & 31, qc = q >> 5;
                    // the pivot column's panel entries, from the lane that holds it
                    float pc[kGjBlock];
#pragma unroll
                    for (int pp = 0; pp < kGjBlock; ++pp) {
                        float mine = P[pp][0];
#pragma unroll
                        for (int cc = 1; cc < kGjCols; ++cc)
                            if (cc == qc) mine = P[pp][cc];
                        pc[pp] = __shfl_sync(kFullMask, mine, ql);
                    }
                    const float inv = __frcp_rn(pc[p]);
#pragma unroll
                    for (int cc = 0; cc < kGjCols; ++cc) {
                        const bool isq = (lane + 32 * cc) == q;
                        if (isq) ucol[cc] = true;
                        const float nk = isq ? inv : P[p][cc] * inv;
#pragma unroll
                        for (int pp = 0; pp < kGjBlock; ++pp)
                            if (pp != p) P[pp][cc] = fmaf(-pc[pp], nk, isq ? 0.0f : P[pp][cc]);
                        P[p][cc] = nk;
                    }
                    if (lane == 0) s_q[k0 + p] = q;
                }
            }
        }
#pragma unroll
        for (int cc = 0; cc < kGjCols; ++cc) {
            const int col = lane + 32 * cc;
            if (col < n) {
                s_used[col] = ucol[cc] ? 1 : 0;
#pragma unroll
                for (int p = 0; p < kGjBlock; ++p)
                    if (p < nb) panel[p][col] = P[p][cc];
            }
        }
    
}

template <int R>
__device__ __forceinline__ void newton_reg_block(const Consts& c, double* __restrict__ J,
                                                 const float* __restrict__ As, const double2* __restrict__ rowinfo,
                                                 const double* __restrict__ F, const XTab* __restrict__ xtab,
                                                 double* __restrict__ coef, const double rho, double* __restrict__ work,
                                                 double* __restrict__ stats, int* __restrict__ status,
                                                 float* __restrict__ Xg, double* __restrict__ Sg,
                                                 int* __restrict__ xstate, const bool xcount, const bool cl) {
    extern __shared__ __align__(16) double dsm[];
    __shared__ __align__(16) float s_colq[2][kColPad];
    __shared__ float s_rowk[2][128];
    __shared__ float s_wc[2][8];
    __shared__ int s_wi[2][8];
    __shared__ int s_q[128];
    __shared__ int s_qinv[128];
    __shared__ double sv[kGjThreads / 32];
    __shared__ int si[kGjThreads / 32];
    __shared__ double s_x[128];
    __shared__ double s_scale[128];
    __shared__ double s_sold[128];
    __shared__ float s_rf[128];
    __shared__ unsigned s_red[2][32];
    __shared__ int s_piv, s_fail, s_done, s_conv, s_reuse;
    __shared__ double s_anorm;
    __shared__ float s_panel[2][kGjBlock][128];                // panel rows of a round (by round parity)
    __shared__ __align__(16) float s_colb[kGjBlock][kColPad];  // the round's pivot columns
    __shared__ unsigned char s_used[128];                      // columns pivoted so far
    const int n = c.n;
    const int ldj = reg_ldj(n);
    if (cl) {
        const unsigned rank = cluster_rank();
        if (rank != 0) {
            newton_residual_rows(n, ldj, J, F, dsm, s_x, s_scale, s_sold, s_rf, &s_red[0][0], rank);
            return;
        }
    }
    double* Js = dsm;                                             // [n][ldj] FP64 copy of J
    float* Xs = reinterpret_cast<float*>(dsm + (size_t)n * ldj);  // [n][n] inverse
    // G groups of R consecutive rows; G * R <= n + R - 1 < kColPad and
    // G * n <= 1024 because the launcher picks R >= n / min(1024 / n, 32)
    const int G = (n + R - 1) / R;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int j = tid % n;
    const int g = tid / n;
    const bool owner = g < G;
    const int i0 = g * R;  // first owned row

    // warp 0: norms of F, ||A||_inf, status
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
            mF = fmax(mF, __shfl_xor_sync(kFullMask, mF, off));
            mS = fmax(mS, __shfl_xor_sync(kFullMask, mS, off));
            an = fmax(an, __shfl_xor_sync(kFullMask, an, off));
        }
        bad = __any_sync(kFullMask, bad);
        if (lane == 0) {
            stats[0] = bad ? INFINITY : mF;
            stats[1] = mS;
            stats[2] = 0.0;
            s_anorm = an;
            s_fail = ((*status) & (kStatusNonfinite | kStatusSingular)) | (bad ? kStatusNonfinite : 0);
            s_done = 0;
        }
    }
    for (int i = tid; i < n; i += kGjThreads) s_scale[i] = rowinfo[i].x;
    if (tid < 64) s_red[tid >> 5][tid & 31] = 0u;  // slots without a warp stay 0
    for (int i = n + tid; i < kColPad; i += kGjThreads) s_colq[0][i] = s_colq[1][i] = 0.0f;  // rows past n
    // J to shared memory: warp w copies rows w, w + 32, ..., its loads all in flight
    // before the stores (no integer division per element)
    for (int i0r = 0; i0r < n; i0r += 4 * (kGjThreads / 32)) {
        double t[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0r + u * (kGjThreads / 32) + warp;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int jj = lane + 32 * v;
                t[u][v] = (i < n && jj < n) ? J[(size_t)i * n + jj] : 0.0;
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0r + u * (kGjThreads / 32) + warp;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int jj = lane + 32 * v;
                if (i < n && jj < n) Js[i * ldj + jj] = t[u][v];
            }
        }
    }
    // (columns 128 .. n - 1 when n > 128 do not occur: this kernel serves n <= 128)
    for (int i = n + tid; i < kColPad; i += kGjThreads)
        for (int p = 0; p < kGjBlock; ++p) s_colb[p][i] = 0.0f;  // rows past n
    if (tid == 0) {
        // try the kept inverse unless the last attempt failed and the update since
        // then is not ten times smaller than the one that preceded that failure
        // (a plan's state, xcount: xstate[4], xstate[5] hold the max |Delta| of the
        // previous step and of the step before the last failed attempt, as FP32
        // bits; 0: none); an attempt that would fail leaves the result unchanged,
        // as the elimination starts afresh
        bool reuse = Xg != nullptr && *xstate == 1;
        if (reuse && xcount) {
            const float dprev = __int_as_float(xstate[4]), dfail = __int_as_float(xstate[5]);
            if (dfail > 0.0f && !(dprev <= 0.1f * dfail)) reuse = false;
        }
        s_reuse = reuse ? 1 : 0;
    }
    if (tid < n) s_x[tid] = 0.0;
    __syncthreads();
    if (s_fail) {
        if (tid == 0) atomicOr(status, s_fail);
        return;
    }
    const double tolfac = 4.0 * sqrt((double)n) * 0x1p-53 * s_anorm;
    int sweeps = 0;
    bool converged = false;
    if (s_reuse) {
        // the previous Newton step's inverse (of its row-scaled matrix) as the
        // approximate inverse; J changes little between late Newton steps
        {
            // 16 values per thread in flight (n <= 128: n^2 <= 16 x 1024)
            float t[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int idx = u * kGjThreads + tid;
                t[u] = idx < n * n ? Xg[idx] : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int idx = u * kGjThreads + tid;
                if (idx < n * n) Xs[idx] = t[u];
            }
        }
        for (int i = tid; i < n; i += kGjThreads) s_sold[i] = Sg[i];
        __syncthreads();
        converged = refine_fp64(n, ldj, Js, Xs, s_sold, s_scale, F, s_x, s_rf, s_red, &s_conv, tolfac, kReuseMax,
                                true, &sweeps, cl) == 1;
        if (xcount && converged && tid == 0) xstate[2] += 1;  // counter of steps that reused the inverse
        if (xcount && !converged && tid == 0) xstate[5] = xstate[4];
    }
    if (!converged) {
        sweeps = 0;  // the reported sweeps are those of the solve that is kept
        if (tid < n) s_x[tid] = 0.0;
        if (tid == 0) s_done = 0;
        float v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = i0 + r;
            v[r] = (owner && i < n) ? As[(size_t)i * n + j] : 0.0f;
        }
        bool used = false;  // this thread's column has been a pivot column
        __syncthreads();
        if constexpr (R % kGjBlock == 0) {
            // Blocked form: rounds of kGjBlock pivots.  The kGjBlock pivot steps of a
            // round on the panel rows k0.. are a block pivot on P = A[K][Q]; for the
            // other rows i they compose to
            //   A[i][j] <- (j in Q ? 0 : A[i][j]) - sum_p A[i][q_p] R_p[j]
            // with the pre-round entries A[i][q_p] and the final panel rows R_p, so a
            // round takes three block barriers instead of two per pivot:
            //   (1) the owners of the panel rows write them to shared memory;
            //   (2) one warp pivots the panel in registers (lane L holds columns
            //       L + 32 c), with shuffles only;
            //   (3) the owners of the round's pivot columns publish them;
            //   (4) every thread updates its rows.
            for (int i = tid; i < 128; i += kGjThreads) s_used[i] = 0;
            __syncthreads();
            int round = 0;
            for (int gs = 0; gs < G; ++gs) {
#pragma unroll
                for (int mb = 0; mb < R / kGjBlock; ++mb, ++round) {
                    const int k0 = gs * R + mb * kGjBlock;
                    if (k0 >= n) break;  // uniform
                    const int nb = min(kGjBlock, n - k0);
                    float(*panel)[128] = s_panel[round & 1];
                    // (1)
                    if (owner && g == gs) {
#pragma unroll
                        for (int p = 0; p < kGjBlock; ++p)
                            if (p < nb) panel[p][j] = v[mb * kGjBlock + p];
                    }
                    __syncthreads();
                    // (2) warp 0 pivots the panel: lane L holds columns L + 32 c
                    if (warp == 0) gj_pivot_panel(panel, k0, nb, n, lane, s_used, s_q, &s_done);
                    __syncthreads();
                    if (s_done != 0) goto elimination_done;  // uniform
                    // (3)
                    int pj = -1;
#pragma unroll
                    for (int p = 0; p < kGjBlock; ++p)
                        if (p < nb && s_q[k0 + p] == j) pj = p;
                    if (owner && pj >= 0) {
                        used = true;
                        float4* dst = reinterpret_cast<float4*>(&s_colb[pj][i0]);
#pragma unroll
                        for (int qq = 0; qq < R / 4; ++qq)
                            dst[qq] = make_float4(v[4 * qq], v[4 * qq + 1], v[4 * qq + 2], v[4 * qq + 3]);
                    }
                    __syncthreads();
                    // (4)
                    if (owner) {
                        float rk[kGjBlock];
#pragma unroll
                        for (int p = 0; p < kGjBlock; ++p) rk[p] = p < nb ? panel[p][j] : 0.0f;
#pragma unroll
                        for (int r = 0; r < R; ++r) v[r] = pj >= 0 ? 0.0f : v[r];
#pragma unroll
                        for (int p = 0; p < kGjBlock; ++p) {
                            const float4* cb = reinterpret_cast<const float4*>(&s_colb[p][i0]);
#pragma unroll
                            for (int qq = 0; qq < R / 4; ++qq) {
                                const float4 m = cb[qq];
                                v[4 * qq + 0] = fmaf(-m.x, rk[p], v[4 * qq + 0]);
                                v[4 * qq + 1] = fmaf(-m.y, rk[p], v[4 * qq + 1]);
                                v[4 * qq + 2] = fmaf(-m.z, rk[p], v[4 * qq + 2]);
                                v[4 * qq + 3] = fmaf(-m.w, rk[p], v[4 * qq + 3]);
                            }
                        }
                        if (g == gs) {
#pragma unroll
                            for (int p = 0; p < kGjBlock; ++p)
                                if (p < nb) v[mb * kGjBlock + p] = rk[p];
                        }
                    }
                }
            }
        } else {
            for (int gs = 0; gs < G; ++gs) {
                // warps that hold threads of group gs
                const int w0 = (gs * n) >> 5;
                const int w1 = (gs * n + n - 1) >> 5;
                const bool in_group_warp = warp >= w0 && warp <= w1;
        #pragma unroll
                for (int rs = 0; rs < R; ++rs) {
                    const int k = gs * R + rs;
                    if (k >= n) break;  // uniform
                    const int b = k & 1;
                    // [A] group gs publishes row k and per-warp candidates over its unused columns
                    if (in_group_warp) {
                        const bool mine = owner && g == gs;
                        float a = -1.0f;
                        int idx = 1 << 30;
                        if (mine) {
                            s_rowk[b][j] = v[rs];
                            if (!used) {
                                a = fabsf(v[rs]);
                                idx = j;
                            }
                        }
        #pragma unroll
                        for (int off = 16; off > 0; off >>= 1) {
                            const float oa = __shfl_xor_sync(kFullMask, a, off);
                            const int oi = __shfl_xor_sync(kFullMask, idx, off);
                            if (oa > a || (oa == a && oi < idx)) {
                                a = oa;
                                idx = oi;
                            }
                        }
                        if (lane == 0) {
                            s_wc[b][warp - w0] = a;
                            s_wi[b][warp - w0] = idx;
                        }
                    }
                    __syncthreads();
                    // [B] pivot column q; its owners publish it
                    float best = s_wc[b][0];
                    int q = s_wi[b][0];
                    for (int w = 1; w <= w1 - w0; ++w) {
                        const float a = s_wc[b][w];
                        const int qi = s_wi[b][w];
                        if (a > best || (a == best && qi < q)) {
                            best = a;
                            q = qi;
                        }
                    }
                    if (!(best > 1e-30f)) {
                        if (tid == 0) s_done = -1;
                        goto elimination_done;  // uniform: every thread read the same candidates
                    }
                    if (tid == 0) s_q[k] = q;
                    if (owner && j == q) {
                        used = true;
        #pragma unroll
                        for (int r = 0; r < R; ++r) s_colq[b][i0 + r] = v[r];
                    }
                    __syncthreads();
                    // [C] eliminate column q from every row but k, scale row k
                    if (owner) {
                        const float inv = 1.0f / s_rowk[b][q];
                        const float nk = (j == q) ? inv : s_rowk[b][j] * inv;
                        if (j == q) {
        #pragma unroll
                            for (int r = 0; r < R; ++r) v[r] = 0.0f;
                        }
                        if (R >= 4) {
                            const float4* col4 = reinterpret_cast<const float4*>(&s_colq[b][i0]);
        #pragma unroll
                            for (int qq = 0; qq < R / 4; ++qq) {
                                const float4 m = col4[qq];
                                v[4 * qq + 0] = fmaf(-m.x, nk, v[4 * qq + 0]);
                                v[4 * qq + 1] = fmaf(-m.y, nk, v[4 * qq + 1]);
                                v[4 * qq + 2] = fmaf(-m.z, nk, v[4 * qq + 2]);
                                v[4 * qq + 3] = fmaf(-m.w, nk, v[4 * qq + 3]);
                            }
                        } else {
        #pragma unroll
                            for (int r = 0; r < R; ++r) v[r] = fmaf(-s_colq[b][i0 + r], nk, v[r]);
                        }
                        if (g == gs) v[rs] = nk;
                    }
                }
            }
        }
    elimination_done:
        __syncthreads();
        // X[q_k][m] = a[k][q_m]
        if (tid < n && s_done == 0) s_qinv[s_q[tid]] = tid;
        __syncthreads();
        if (owner && s_done == 0) {
            const int m = s_qinv[j];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int i = i0 + r;
                if (i < n) Xs[s_q[i] * n + m] = v[r];
            }
        }
        __syncthreads();
        if (s_done == 0) {
            converged = refine_fp64(n, ldj, Js, Xs, s_scale, s_scale, F, s_x, s_rf, s_red, &s_conv, tolfac,
                                    kRefineMax, false, &sweeps, cl) == 1;
            // keep an inverse that worked for the next Newton step
            if (Xg != nullptr) {
                if (converged) {
                    for (int idx = tid; idx < n * n; idx += kGjThreads) Xg[idx] = Xs[idx];
                    for (int i = tid; i < n; i += kGjThreads) Sg[i] = s_scale[i];
                }
                if (tid == 0) {
                    *xstate = converged ? 1 : 0;
                    if (xcount) xstate[1] += 1;  // counter of eliminations
                }
            }
        } else if (Xg != nullptr && tid == 0) {
            *xstate = 0;
        }
    }
    double* xres = work + n;
    if (converged) {
        if (tid < n) xres[tid] = s_x[tid];
        __syncthreads();
    } else {
        for (int i = tid; i < n; i += kGjThreads) work[i] = F[i];
        __syncthreads();
        lu_fp64_block(n, J, work, xres, &s_fail, &s_piv, sv, si);
        __syncthreads();
    }
    if (s_fail) {
        if (tid == 0) atomicOr(status, s_fail);
        return;
    }
    if (warp == 0) {
        double mD = 0.0;
        bool bad = false;
        for (int i = lane; i < n; i += 32) {
            mD = fmax(mD, fabs(xres[i]));
            bad |= !isfinite(xres[i]);
        }
        for (int off = 16; off > 0; off >>= 1) mD = fmax(mD, __shfl_xor_sync(kFullMask, mD, off));
        bad = __any_sync(kFullMask, bad);
        if (lane == 0) {
            stats[2] = mD;
            stats[3] = converged ? (double)sweeps : -1.0;
            if (bad) s_fail = kStatusNonfinite;
            if (Xg != nullptr && xcount) xstate[4] = __float_as_int((float)mD);
        }
    }
    __syncthreads();
    if (s_fail) {
        if (tid == 0) atomicOr(status, s_fail);
        return;
    }
    for (int i = tid; i < n; i += kGjThreads) coef[i] = fma(-rho, xres[i], coef[i]);
}

template <int R>
__global__ void __launch_bounds__(kGjThreads) k_newton_reg(const Consts c, double* __restrict__ J,
                                                           const float* __restrict__ As,
                                                           const double2* __restrict__ rowinfo,
                                                           const double* __restrict__ F,
                                                           const XTab* __restrict__ xtab, double* __restrict__ coef,
                                                           double rho, double* __restrict__ work,
                                                           double* __restrict__ stats, int* __restrict__ status,
                                                           float* __restrict__ Xinv, double* __restrict__ Sinv,
                                                           int* __restrict__ xstate) {
    // a plan's xstate word is followed by its two solver counters and the two words
    // of the reuse gate; launched as a cluster (n > 64), CTA 0 solves and every CTA
    // forms 16 rows of each residual
    const bool cl = cluster_ctas() > 1;
    newton_reg_block<R>(c, J, As, rowinfo, F, xtab, coef, rho, work, stats, status, Xinv, Sinv, xstate, true, cl);
    if (cl && cluster_rank() == 0) {
        // the stop round: the other CTAs read the command, and none leaves while
        // another may still read its shared memory
        __syncthreads();
        if (threadIdx.x >= 1 && threadIdx.x < cluster_ctas()) cluster_st_s32(cluster_addr(&s_ncmd[0], threadIdx.x), 0);
        cluster_barrier();  // (1)
        cluster_barrier();  // (2)
    }
}

// One block per problem of a batch; afterwards thread 0 advances the problem's
// iteration state: a failed step ends it (result -2 singular, -1 non-finite),
// and so does a dimensionless residual on entry below tol (result 1, converged,
// update applied).
template <int R>
__global__ void __launch_bounds__(kGjThreads) k_newton_reg_batched(BatchProblem* __restrict__ P,
                                                                   double* __restrict__ coef_base, double tol,
                                                                   double rho_relax, int n_relax,
                                                                   int* __restrict__ n_active) {
    BatchProblem& B = P[blockIdx.x];
    if (!B.active) return;
    const double rho = B.iter < n_relax ? rho_relax : 1.0;
    newton_reg_block<R>(B.t.c, B.J, B.As, B.rowinfo, B.F, B.xtab, coef_base + B.coef_off, rho, B.work, B.stats,
                        B.status, B.Xinv, B.Sinv, &B.xstate, false, false);
    __syncthreads();
    if (threadIdx.x == 0) {
        B.iter += 1;
        const int stw = *B.status;
        int res = 0;
        if (stw & kStatusSingular) res = -2;
        else if (stw & kStatusNonfinite) res = -1;
        else if (B.stats[1] < tol) res = 1;
        if (res != 0) {
            B.result = res;
            B.active = 0;
            atomicSub(n_active, 1);
        }
    }
}

// ------------------------------------------------------------------------
__global__ void k_dressing(const Consts c, const double* __restrict__ coef, int n, const double* __restrict__ x,
                           double* __restrict__ lG, double* __restrict__ lZ, int* __restrict__ status) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    const double xm = x[m];
    if (!(xm > 0.0)) {
        lG[m] = lZ[m] = NAN;
        atomicOr(status, kStatusNonfinite);
        return;
    }
    double g, z;
    dressing_eval(c, coef, coef + c.NZ, xm, g, z, nullptr);
    lG[m] = g;
    lZ[m] = z;
}

// Schwinger function (Sec. 2.2, Sec. 5): nodes in u = ln p^2 over
// [ln eps2, ln lambda2], p = e^{u/2}, d|p| = (p/2) du.
__global__ void k_schwinger_map(const Consts c, int n, const double* __restrict__ gx, const double* __restrict__ gw,
                                double* __restrict__ pn, double* __restrict__ wn) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double u = c.L0 + c.L1 * gx[i];
    const double p = exp(0.5 * u);
    pn[i] = p;
    wn[i] = c.L1 * gw[i] * 0.5 * p;
}

// sigw_n = w_n Z(p_n^2) / (pi p_n^2)
__global__ void k_schwinger_weights(const Consts c, const double* __restrict__ coef, int n,
                                    const double* __restrict__ pn, const double* __restrict__ wn,
                                    double* __restrict__ sigw) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double p = pn[i];
    const double x = p * p;
    double g, z;
    dressing_eval(c, coef, coef + c.NZ, x, g, z, nullptr);
    sigw[i] = wn[i] * exp(z) / x / kPi;
}

// cos x for |x| < 2^49 (the caller takes the library cos beyond), FP64-accurate (a
// few units in the last place) with most of the arithmetic on the FP32 pipe.  Cody-Waite reduction (Cody & Waite 1980):
// k = nearest integer to 2x/pi (the 1.5 2^52 shifter; below |x| = 2^18 an integer
// within 0.52 of 2x/pi from FP32 arithmetic), r = x - k pi/2 with pi/2 in two FP64
// parts (FMA; P1 = pi/2 rounded to FP64, P2 = pi/2 - P1 rounded; the remainder
// |pi/2 - P1 - P2| < 1.5e-33 leaves k below 2^50 an error under 2e-18, below an ulp
// of r), |r| <= pi/4 (+ 0.031 below 2^18).  Then by the quadrant k mod 4
// cos x = +-cos r or -+sin r, with the Taylor series split as
//   cos r = (1 - r^2/2) + r^4 (1/4! - r^2/6! + ... + r^14/18!)
//   sin r = (r - r^3/6) + r^5 (1/5! - r^2/7! + ... + r^14/19!)
// (truncation below 1e-20 for |r| <= pi/4 + 0.031): the leading terms in FP64, the
// tails (at most 0.019) in double-float, both tails for every lane so that the quadrant
// selects without divergence.  The caller keeps the two parts apart (an FP64 sum of
// w lead, a double-float sum of w tail) and adds them once at the end.
constexpr double kPio2_1 = 1.5707963267948966;
constexpr double kPio2_2 = 6.123233995736766e-17;
constexpr double kTwoOverPi = 0.6366197723675814;
constexpr double kRoundShifter = 6755399441055744.0;  // 1.5 2^52
constexpr unsigned kCosReduceMaxHi = 0x43000000u;  // high word of 2^49: from there the library cos
constexpr unsigned kCosFastHi = 0x41100000u;       // high word of 2^18: below it, k from FP32
constexpr float kTwoOverPiF = 0.636619772f;        // 2/pi rounded to FP32

// The leading 24 significant bits of x as an FP32 number (truncated toward zero;
// 0 below the FP32 normal range), by integer operations on its bits (|x| < 2^18).
__device__ __forceinline__ float lead24(double x) {
    const unsigned hb = (unsigned)__double2hiint(x), lb = (unsigned)__double2loint(x);
    const int e = (int)((hb >> 20) & 0x7ffu) - 896;  // biased FP32 exponent
    if (e < 1) return 0.0f;
    return __int_as_float((int)((hb & 0x80000000u) | ((unsigned)e << 23) | ((hb & 0xfffffu) << 3) | (lb >> 29)));
}


struct CosTail { float2 c[8], s[8]; };

// Taylor tail coefficients (-1)^k / (2k + 4)! and (-1)^k / (2k + 5)!, k = 0..7, as
// double-float pairs of the FP64 quotients
__device__ __forceinline__ CosTail cos_tail_coefficients() {
    CosTail t;
    double fc = 24.0, fs = 120.0;  // (2k + 4)!, (2k + 5)!
    for (int k = 0; k < 8; ++k) {
        const double sg = (k & 1) ? -1.0 : 1.0;
        t.c[k] = df_split(sg / fc, 0);
        t.s[k] = df_split(sg / fs, 0);
        fc *= (double)((2 * k + 5) * (2 * k + 6));
        fs *= (double)((2 * k + 6) * (2 * k + 7));
    }
    return t;
}

struct CosParts { double lead; float2 tail; };

__device__ __forceinline__ CosParts cos_df(double x, const CosTail& T) {
    int k;
    double kd;
    if (((unsigned)__double2hiint(x) & 0x7fffffffu) < kCosFastHi) {
        // |x| < 2^18: k from the FP32 product of the leading 24 bits of x and 2/pi,
        // rounded by the 1.5 2^23 shifter (within 0.02 of x 2/pi, so |r| <= pi/4 +
        // 0.031, where the truncated series keep their accuracy), and its double by
        // integer operations: no FP64 instruction
        k = __float_as_int(fmaf(lead24(x), kTwoOverPiF, 12582912.0f)) - 0x4b400000;
        kd = int_as_double(k);
    } else {
        kd = fma(x, kTwoOverPi, kRoundShifter);
        k = __double2loint(kd);
        kd -= kRoundShifter;
    }
    const int q = k & 3;
    double r = fma(-kd, kPio2_1, x);
    r = fma(-kd, kPio2_2, r);
    const double r2 = r * r;
    const float2 rd = df_split(r, 0);
    const float2 r2d = df_mul(rd, rd);
    const float2 r4d = df_mul(r2d, r2d);
    float2 pc = T.c[7], ps = T.s[7];
#pragma unroll
    for (int k = 6; k >= 0; --k) {
        pc = df_muladd(pc, r2d, T.c[k]);
        ps = df_muladd(ps, r2d, T.s[k]);
    }
    const bool odd = (q & 1) != 0;
    float2 t = df_mul(odd ? ps : pc, r4d);
    t = df_mul(t, odd ? rd : make_float2(1.0f, 0.0f));
    // leading terms as one FMA, P + P k with P = +-r (odd) or +-1 (even) and
    // k = -r^2/6 or -r^2/2; the sign of the quadrant goes into P's sign bit
    const bool neg = (q == 1 || q == 2);
    const double base = odd ? r : 1.0;
    const double P = __hiloint2double(__double2hiint(base) ^ (neg ? (int)0x80000000 : 0), __double2loint(base));
    CosParts o;
    o.lead = fma(P, r2 * (odd ? -1.0 / 6.0 : -0.5), P);
    o.tail = neg ? make_float2(-t.x, -t.y) : t;
    return o;
}

// partial[s][m] = sum over nodes of split s of sigw_n cos(t_m p_n).
// Block: kSchT times x kSchPh phases; nodes staged through shared memory.
constexpr int kSchT = 32;
constexpr int kSchPh = 8;
constexpr int kSchTile = 512;

__global__ void __launch_bounds__(kSchT * kSchPh) k_schwinger_sum(int n_nodes, const double* __restrict__ pn,
                                                                  const double* __restrict__ sigw,
                                                                  const double* __restrict__ t, int n_t,
                                                                  int nsplit, double* __restrict__ partial) {
    __shared__ double sp[kSchTile];
    __shared__ double sw[kSchTile];
    __shared__ float2 swd[kSchTile];  // the weights as double-float pairs
    __shared__ double sred[kSchPh][kSchT];
    const int tl = threadIdx.x % kSchT;
    const int ph = threadIdx.x / kSchT;
    const int m = blockIdx.x * kSchT + tl;
    const int s = blockIdx.y;
    const int per = (n_nodes + nsplit - 1) / nsplit;
    const int n0 = s * per;
    const int n1 = min(n_nodes, n0 + per);
    const double tm = m < n_t ? t[m] : 0.0;
    // Scale of the double-float tail sum: the largest |w| of the split maps to
    // about 2^100, so that w tail (|tail| <= 0.016) summed over up to 2^20 nodes
    // stays inside the FP32 range, and weights more than 2^-226 below the largest
    // (whose tail terms are below 2^-232 of it) are the only ones flushed.
    __shared__ int semax[kSchPh];
    int em = 0;
    for (int q = n0 + (int)threadIdx.x; q < n1; q += kSchT * kSchPh)
        em = max(em, (int)(((unsigned)__double2hiint(sigw[q]) >> 20) & 0x7ffu));
    em = (int)__reduce_max_sync(kFullMask, (unsigned)em);
    if (tl == 0) semax[ph] = em;
    __syncthreads();
    em = semax[0];
#pragma unroll
    for (int q = 1; q < kSchPh; ++q) em = max(em, semax[q]);
    const int sh = em - 1123;  // biased FP32 exponent of (largest |w|) 2^-sh is 227
    const CosTail T = cos_tail_coefficients();
    double acc = 0.0;                   // sum of w lead (FP64)
    float2 acct = make_float2(0.f, 0.f);  // sum of w tail 2^-sh (double-float)
    for (int base = n0; base < n1; base += kSchTile) {
        const int cnt = min(kSchTile, n1 - base);
        for (int q = threadIdx.x; q < cnt; q += kSchT * kSchPh) {
            sp[q] = pn[base + q];
            const double w = sigw[base + q];
            sw[q] = w;
            swd[q] = df_split(w, sh);
        }
        __syncthreads();
#pragma unroll 2
        for (int q = ph; q < cnt; q += kSchPh) {
            const double x = tm * sp[q];
            CosParts cp = cos_df(x, T);
            // |x| >= 2^49 (or not finite), from the exponent field: beyond the two-part reduction
            if (((unsigned)__double2hiint(x) & 0x7fffffffu) >= kCosReduceMaxHi) {
                cp.lead = cos(x);
                cp.tail = make_float2(0.f, 0.f);
            }
            acc = fma(sw[q], cp.lead, acc);
            df_fma(acct, swd[q], cp.tail);
            df_renorm(acct);
        }
        __syncthreads();
    }
    acc += df_widen(acct.x, 1023 + sh) + df_widen(acct.y, 1023 + sh);
    sred[ph][tl] = acc;
    __syncthreads();
    if (ph == 0 && m < n_t) {
        double v = 0.0;
        for (int q = 0; q < kSchPh; ++q) v += sred[q][tl];
        partial[(size_t)s * n_t + m] = v;
    }
}

__global__ void k_schwinger_reduce(int n_t, int nsplit, const double* __restrict__ partial,
                                   double* __restrict__ delta, int* __restrict__ status) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n_t) return;
    double v = 0.0;
    for (int s = 0; s < nsplit; ++s) v += partial[(size_t)s * n_t + m];
    delta[m] = v;
    if (!isfinite(v)) atomicOr(status, kStatusNonfinite);
}

inline int blocks_for(long long n, int bs) { return (int)((n + bs - 1) / bs); }

}  // namespace

cudaError_t launch_gauss_legendre(int n, double* inv, double* x, double* w, cudaStream_t s) {
    // inv: n + 2 doubles of scratch for the table 1/k used by the recurrence
    k_inverse_table<<<blocks_for(n + 1, 256), 256, 0, s>>>(n, inv);
    k_gauss_legendre<<<blocks_for((n + 1) / 2, 128), 128, 0, s>>>(n, inv, x, w);
    return cudaGetLastError();
}

cudaError_t launch_setup_rules(const Consts& c, const double* gl_r, const double* gw_r, const double* gl_a,
                               const double* gw_a, Rad* rad, Ang* ang, double* theta, double* xcol, Row* rows,
                               int Rt, cudaStream_t s) {
    const long long total = (long long)rad_entries(c) + c.na + c.Rc + Rt;
    k_setup_rules<<<blocks_for(total, 128), 128, 0, s>>>(c, gl_r, gw_r, gl_a, gw_a, rad, ang, theta, xcol, rows, Rt);
    return cudaGetLastError();
}

cudaError_t launch_tables(const Consts& c, const double* coef, const Rad* rad, const double* xcol, YTab* ytab,
                          double* phiy, XTab* xtab, double* phix, cudaStream_t s) {
    k_tables<<<blocks_for((long long)rad_entries(c) + c.Rc, 64), 64, 0, s>>>(c, coef, rad, xcol, ytab, phiy, xtab, phix);
    return cudaGetLastError();
}

cudaError_t launch_rowreduce(bool full, const Consts& c, int Rt, int KS, int nch, const Rad* rad, const Ang* ang,
                             const Row* rows, const YTab* ytab, const double* phiy, const double* Upart,
                             const double* Vpart, double* D, cudaStream_t s) {
    (void)Rt;
    const dim3 grid(c.Rc + 2, full ? (c.N + kRowJ - 1) / kRowJ : 1);
    if (full)
        k_rowreduce<true><<<grid, kRowBlock, 0, s>>>(c, Rt, KS, nch, rad, ang, rows, ytab, phiy, Upart, Vpart, D);
    else
        k_rowreduce<false><<<grid, kRowBlock, 0, s>>>(c, Rt, KS, nch, rad, ang, rows, ytab, phiy, Upart, Vpart, D);
    return cudaGetLastError();
}

// ---- Newton iteration as a device-driven loop (the body of a CUDA-graph while node)
__global__ void k_solve_begin(SolveCtl* __restrict__ ctl, double tol, int max_steps, const double* __restrict__ src,
                              double* __restrict__ dst, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
    if (threadIdx.x == 0) {
        ctl->tol = tol;
        ctl->max_steps = max_steps;
        ctl->steps = 0;
        ctl->status = 0;
        ctl->converged = 0;
    }
}

// The stopping rule of the host loop: a status word set by any kernel of the
// step, the dimensionless residual below tol (a NaN never is), or the step limit.
__global__ void k_solve_decide(SolveCtl* __restrict__ ctl, const double* __restrict__ stats,
                               const int* __restrict__ status, cudaGraphConditionalHandle cond) {
    const int steps = ctl->steps + 1;
    const int st = *status;
    const bool conv = st == 0 && stats[1] < ctl->tol;
    ctl->steps = steps;
    ctl->status = st;
    ctl->converged = conv ? 1 : 0;
    for (int k = 0; k < 4; ++k) ctl->stats[k] = stats[k];
    cudaGraphSetConditional(cond, (st != 0 || conv || steps >= ctl->max_steps) ? 0u : 1u);
}

__global__ void k_copy_vector(const double* __restrict__ src, double* __restrict__ dst, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

cudaError_t launch_solve_begin(SolveCtl* ctl, double tol, int max_steps, const double* src, double* dst, int n,
                               cudaStream_t s) {
    k_solve_begin<<<1, 256, 0, s>>>(ctl, tol, max_steps, src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_solve_decide(SolveCtl* ctl, const double* stats, const int* status,
                                cudaGraphConditionalHandle cond, cudaStream_t s) {
    k_solve_decide<<<1, 1, 0, s>>>(ctl, stats, status, cond);
    return cudaGetLastError();
}

cudaError_t launch_solve_end(const double* src, double* dst, int n, cudaStream_t s) {
    k_copy_vector<<<1, 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_assemble(bool full, const Consts& c, const XTab* xtab, const double* phix, const double* D,
                            double* J, double* F, int* status, cudaStream_t s) {
    const long long total = (full ? (long long)c.n * c.n : 0) + c.n;
    const int nb = blocks_for(total, 256);
    if (full) k_assemble<true><<<nb, 256, 0, s>>>(c, xtab, phix, D, J, F, status);
    else k_assemble<false><<<nb, 256, 0, s>>>(c, xtab, phix, D, J, F, status);
    return cudaGetLastError();
}

bool lu_scales_rows(int n, bool lu32) { return n <= 128 || (n > kGjMaxN && lu32 && n <= 2 * DSE_MAX_CHEB); }

cudaError_t launch_assemble_scale(const Consts& c, const XTab* xtab, const double* phix, const double* D, double* J,
                                  double* F, float* As, double2* rowinfo, int* status, cudaStream_t s) {
    k_assemble_scale<<<c.n, kScaleThreads, 0, s>>>(c, xtab, phix, D, J, F, As, rowinfo, status);
    return cudaGetLastError();
}

// The Newton-step kernel for n <= 128: as a cluster of ceil(n / 16) CTAs (one per
// SM; the residual of each refinement sweep shared out by rows) when n exceeds
// DSE_NEWTON_CLUSTER_MIN_N and this GPU can place such a cluster, else one CTA.
#ifndef DSE_NEWTON_CLUSTER_MIN_N
#define DSE_NEWTON_CLUSTER_MIN_N 65
#endif
size_t newton_reg_smem(int n) { return sizeof(double) * (size_t)n * reg_ldj(n) + sizeof(float) * (size_t)n * n; }
int newton_reg_rows(int n) {
    const int G = kGjThreads / n < 32 ? kGjThreads / n : 32;  // same as in the kernel
    const int R = (n + G - 1) / G;
    return R <= 1 ? 1 : R <= 2 ? 2 : R <= 4 ? 4 : R <= 8 ? 8 : 16;
}

// The launch configuration of k_newton_reg<R> for n unknowns; whether a cluster of
// that size can be placed is asked once per kernel and size (prepare_newton_step
// asks it outside any graph capture) and kept.
template <int R>
cudaError_t newton_reg_config(int n, cudaStream_t s, cudaLaunchConfig_t& cfg, cudaLaunchAttribute* at) {
    static int placeable[9] = {-1, -1, -1, -1, -1, -1, -1, -1, -1};
    const size_t smem = newton_reg_smem(n);
    cudaError_t e = cudaFuncSetAttribute(k_newton_reg<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cfg = cudaLaunchConfig_t{};
    cfg.blockDim = dim3(kGjThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.gridDim = dim3(1);
    const int ncta = (n + 15) / 16;
    if (n >= DSE_NEWTON_CLUSTER_MIN_N && ncta > 1 && ncta <= 8) {
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)ncta;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(ncta);
        cfg.attrs = at;
        cfg.numAttrs = 1;
        if (placeable[ncta] < 0) {
            int nclusters = 0;
            if (cudaOccupancyMaxActiveClusters(&nclusters, k_newton_reg<R>, &cfg) != cudaSuccess) {
                cudaGetLastError();
                nclusters = 0;
            }
            placeable[ncta] = nclusters > 0 ? 1 : 0;
        }
        if (placeable[ncta] != 1) {
            cfg.gridDim = dim3(1);
            cfg.attrs = nullptr;
            cfg.numAttrs = 0;
        }
    }
    return cudaSuccess;
}

template <int R>
cudaError_t launch_newton_reg(int n, cudaStream_t s, const Consts& c, double* J, const float* As,
                              const double2* rowinfo, const double* F, const XTab* xtab, double* coef, double rho,
                              double* work, double* stats, int* status, float* Xinv, double* Sinv, int* xstate) {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[1];
    cudaError_t e = newton_reg_config<R>(n, s, cfg, at);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cfg, k_newton_reg<R>, c, J, As, rowinfo, F, xtab, coef, rho, work, stats, status,
                              Xinv, Sinv, xstate);
}

cudaError_t prepare_newton_step(int n) {
    if (n > 128) return cudaSuccess;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[1];
    switch (newton_reg_rows(n)) {
        case 1: return newton_reg_config<1>(n, 0, cfg, at);
        case 2: return newton_reg_config<2>(n, 0, cfg, at);
        case 4: return newton_reg_config<4>(n, 0, cfg, at);
        case 8: return newton_reg_config<8>(n, 0, cfg, at);
        default: return newton_reg_config<16>(n, 0, cfg, at);
    }
}

cudaError_t launch_lu_newton(const Consts& c, double* J, const double* F, const XTab* xtab, double* coef, double rho,
                             double* work, float* As, double2* rowinfo, double* stats, int* status, cudaStream_t s,
                             float* Xinv, double* Sinv, int* xstate, int* done, bool prescaled) {
    if (!Xinv || !Sinv || !xstate) Xinv = nullptr, Sinv = nullptr, xstate = nullptr;
    const int n = c.n;
    cudaError_t e = cudaSuccess;
    if (n <= 128) {
        if (!prescaled) k_scale_rows<<<n, kScaleThreads, 0, s>>>(n, J, As, rowinfo, status);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
#define DSE_LAUNCH_REG(RR) \
    e = launch_newton_reg<RR>(n, s, c, J, As, rowinfo, F, xtab, coef, rho, work, stats, status, Xinv, Sinv, xstate);
        switch (newton_reg_rows(n)) {
            case 1: DSE_LAUNCH_REG(1) break;
            case 2: DSE_LAUNCH_REG(2) break;
            case 4: DSE_LAUNCH_REG(4) break;
            case 8: DSE_LAUNCH_REG(8) break;
            default: DSE_LAUNCH_REG(16) break;
        }
#undef DSE_LAUNCH_REG
        if (e != cudaSuccess) return e;
    } else if (n <= kGjMaxN) {
        const size_t smem = sizeof(float) * (size_t)n * 2 * n;
        e = cudaFuncSetAttribute(k_newton_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_newton_mixed<<<1, kGjThreads, smem, s>>>(c, J, F, xtab, coef, rho, work, stats, status);
    } else {
        if (done && n <= 2 * DSE_MAX_CHEB) {
            if (!prescaled) k_scale_rows<<<n, kScaleThreads, 0, s>>>(n, J, As, rowinfo, status);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = launch_newton_lu32(c, J, As, rowinfo, F, xtab, coef, rho, stats, status, done, s);
            if (e != cudaSuccess) return e;
        } else {
            done = nullptr;
        }
        k_lu_newton<<<1, kLuThreads, 0, s>>>(c, J, F, xtab, coef, rho, work, stats, status, done);
    }
    return cudaGetLastError();
}

cudaError_t launch_dressing(const Consts& c, const double* coef, int n, const double* x, double* lG, double* lZ,
                            int* status, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_dressing<<<blocks_for(n, 128), 128, 0, s>>>(c, coef, n, x, lG, lZ, status);
    return cudaGetLastError();
}

cudaError_t launch_schwinger_map(const Consts& c, int n, const double* gx, const double* gw, double* pn, double* wn,
                                 cudaStream_t s) {
    k_schwinger_map<<<blocks_for(n, 128), 128, 0, s>>>(c, n, gx, gw, pn, wn);
    return cudaGetLastError();
}

// Node splits of the Schwinger sum: as many as fill one wave of resident blocks
// (tb time blocks x splits <= SMs x blocks per SM), so that no SM runs a block
// more than another; at least one split and at least one tile of nodes per split.
// When the time blocks alone exceed a wave: about four blocks per SM.
int schwinger_splits(int n_t, int n_nodes) {
    const int tb = (n_t + kSchT - 1) / kSchT;
    int dev = 0, nsm = 152, occ = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_schwinger_sum, kSchT * kSchPh, 0) != cudaSuccess ||
        occ < 1)
        occ = 1;
    const int slots = nsm * occ;
    int ns = tb > 0 ? slots / tb : 1;
    if (ns < 1) ns = (4 * nsm + tb - 1) / (tb > 0 ? tb : 1);
    const int maxs = (n_nodes + kSchTile - 1) / kSchTile;
    if (ns > maxs) ns = maxs;
    if (ns < 1) ns = 1;
    return ns;
}

cudaError_t launch_schwinger(const Consts& c, const double* coef, int n_nodes, const double* pn, const double* wn,
                             double* sigw, const double* t, int n_t, double* partial, int nsplit, double* delta,
                             int* status, cudaStream_t s) {
    k_schwinger_weights<<<blocks_for(n_nodes, 128), 128, 0, s>>>(c, coef, n_nodes, pn, wn, sigw);
    if (n_t <= 0) return cudaGetLastError();
    const dim3 grid((n_t + kSchT - 1) / kSchT, nsplit);
    k_schwinger_sum<<<grid, kSchT * kSchPh, 0, s>>>(n_nodes, pn, sigw, t, n_t, nsplit, partial);
    k_schwinger_reduce<<<blocks_for(n_t, 256), 256, 0, s>>>(n_t, nsplit, partial, delta, status);
    return cudaGetLastError();
}

cudaError_t launch_series_init(const Consts& c, double2* tq, double* cst, SeriesRec* tab, cudaStream_t s) {
    k_series_init<<<c.sM, 64, 0, s>>>(c, tq, cst, tab);
    return cudaGetLastError();
}

cudaError_t launch_series_table(const Consts& c, const double* coef, const double2* tq, const double* cst,
                                SeriesRec* tab, cudaStream_t s) {
    k_series_table<<<c.sM, kSeriesDotThreads, 0, s>>>(c, coef, tq, cst, tab);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------
// Batched launchers: grid dimension y (z for the row contraction) runs over the
// problems of the batch.
cudaError_t launch_series_table_batched(const BatchProblem* P, int nb, const double* coef_base, cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    k_series_table_batched<<<dim3(kSeriesM / kSeriesIntervalsPerBlock, nb), kSeriesThreads, 0, s>>>(P, coef_base);
    return cudaGetLastError();
}

cudaError_t launch_tables_batched(const BatchProblem* P, int nb, int max_units, const double* coef_base,
                                  cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    const dim3 grid(blocks_for(max_units, 64), nb);
    k_tables_batched<<<grid, 64, 0, s>>>(P, coef_base);
    return cudaGetLastError();
}

cudaError_t launch_rowreduce_batched(bool full, const BatchProblem* P, int nb, int max_rows, int maxN,
                                     cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    const dim3 grid(max_rows, full ? (maxN + kRowJ - 1) / kRowJ : 1, nb);
    if (full) k_rowreduce_batched<true><<<grid, kRowBlock, 0, s>>>(P);
    else k_rowreduce_batched<false><<<grid, kRowBlock, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_assemble_batched(bool full, const BatchProblem* P, int nb, double* J_base, double* F_base,
                                    cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    const dim3 grid(16, nb);
    if (full) k_assemble_batched<true><<<grid, 256, 0, s>>>(P, J_base, F_base);
    else k_assemble_batched<false><<<grid, 256, 0, s>>>(P, J_base, F_base);
    return cudaGetLastError();
}

cudaError_t prepare_newton_batched(int max_n) {
    if (max_n > 128) return cudaErrorInvalidValue;
    const size_t smem = sizeof(double) * (size_t)max_n * reg_ldj(max_n) + sizeof(float) * (size_t)max_n * max_n;
    return cudaFuncSetAttribute(k_newton_reg_batched<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_newton_batched(const BatchProblem* P, int nb, int max_n, double* coef_base, double tol,
                                  double rho_relax, int n_relax, int* n_active, cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    if (max_n > 128) return cudaErrorInvalidValue;
    k_scale_rows_batched<<<dim3(max_n, nb), kScaleThreads, 0, s>>>(P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // R = 16 serves every n <= 128: G = ceil(n/16) <= 8 groups, G n <= 1024 threads;
    // the shared-memory limit was set by prepare_newton_batched (this launch may
    // be captured into a graph)
    const size_t smem = sizeof(double) * (size_t)max_n * reg_ldj(max_n) + sizeof(float) * (size_t)max_n * max_n;
    k_newton_reg_batched<16><<<nb, kGjThreads, smem, s>>>(const_cast<BatchProblem*>(P), coef_base, tol, rho_relax,
                                                           n_relax, n_active);
    return cudaGetLastError();
}

}  // namespace dse
