// dse_series.cuh -- device evaluation of the dressing functions (arXiv:1206.1779
// Sec. 3 Chebyshev expansion of ln G, ln Z in s(x); Sec. 2 IR/UV continuation).
#pragma once

#include "dse_internal.cuh"

namespace dse {

// s(x) = (ln x - L0)/L1 clamped to [-1, 1]; ln G, ln Z and optionally
// phi_j(x) = d ln G/d b_j = d ln Z/d a_j (1/2 for j = 0, T_j(s) otherwise) for
// j < N = max(NZ, NG).  a: the NZ coefficients of ln Z, b: the NG of ln G.
__device__ __forceinline__ void dressing_eval(const Consts& c, const double* __restrict__ a,
                                              const double* __restrict__ b, double x, double& lG,
                                              double& lZ, double* __restrict__ phi) {
    const double lx = log(x);
    double s = (lx - c.L0) * c.invL1;
    s = fmin(1.0, fmax(-1.0, s));
    double g = 0.5 * b[0], zz = 0.5 * a[0];
    if (phi) phi[0] = 0.5;
    if (c.N > 1) {
        if (c.NG > 1) g = fma(b[1], s, g);
        if (c.NZ > 1) zz = fma(a[1], s, zz);
        if (phi) phi[1] = s;
    }
    double t0 = 1.0, t1 = s;
    const double s2 = 2.0 * s;
    for (int j = 2; j < c.N; ++j) {
        const double t2 = fma(s2, t1, -t0);
        t0 = t1;
        t1 = t2;
        if (j < c.NG) g = fma(b[j], t2, g);
        if (j < c.NZ) zz = fma(a[j], t2, zz);
        if (phi) phi[j] = t2;
    }
    if (c.extrap == 0) {
        if (x < c.eps2) {
            // Z = A x^{2 kappa}, G = B x^{-kappa}, matched at eps2
            const double r = lx - c.ln_eps2;
            g = fma(-c.kappa, r, g);
            zz = fma(2.0 * c.kappa, r, zz);
        } else if (x > c.lam2) {
            // G = G_UV [omega ln(x/lambda2) + 1]^delta, Z = Z_UV [...]^gamma
            const double L = log1p(c.omega * (lx - c.ln_lam2));
            g = fma(c.delta, L, g);
            zz = fma(c.gam, L, zz);
        }
    }
    lG = g;
    lZ = zz;
}

}  // namespace dse
