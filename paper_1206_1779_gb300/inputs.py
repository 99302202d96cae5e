"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module only defines workloads: the physical parameters the paper uses
(arXiv:1206.1779 Sec. 2.1 and Sec. 3), the quadrature sizes of each workload,
a smooth starting guess with a seeded perturbation, and seeded Euclidean times
for the Schwinger function.  It holds none of the residual, kernel or Jacobian
arithmetic; both the CUDA path and the CPU oracle receive its outputs as inputs.
"""
from __future__ import annotations

import math

import numpy as np

# Paper values: alpha(mu^2) = 1 with N_c = 3 gives g^2 N_c = 4 pi * 3 (Sec. 2.1);
# Z(x_Z) = 0.256 at x_Z = Lambda^2, x_G = 0 and G(x_G)^{-1} = 0 for the scaling
# solution (Sec. 2.1); delta = -9/44 (Sec. 2); kappa = (93 - sqrt(1201))/98,
# the closed form of the printed 0.595353 (Sec. 2).
KAPPA = (93.0 - math.sqrt(1201.0)) / 98.0
DELTA = -9.0 / 44.0
G2NC = 12.0 * math.pi

WORKLOADS = {
    # one FP64 Newton step: N = 16 per function, 64 radial x 32 angular nodes
    "newton_step_n16": dict(n_cheb=16, n_radial=64, n_angular=32),
    # FP64 full solve + Schwinger function: N = 64, 256 x 128 nodes
    "full_solve_n64": dict(n_cheb=64, n_radial=256, n_angular=128),
    # N = 128 with 512 x 256 nodes
    "matrix_n128": dict(n_cheb=128, n_radial=512, n_angular=256),
}


def problem(n_cheb: int, n_radial: int, n_angular: int, eps2: float = 1e-6, lambda2: float = 1e6,
            g2nc: float = G2NC, x_G: float = 0.0, ginv_G: float = 0.0, x_Z: float | None = None,
            zinv_Z: float = 1.0 / 0.256, kappa: float = KAPPA, delta: float = DELTA,
            radial_mode: int = 0, extrap_mode: int = 0, precision: int = 0, n_cheb_G: int = 0,
            angular_mode: int = 0) -> dict:
    """Problem parameters as a plain dict (field names of dse_problem).  n_cheb is
    the order N_Z of ln Z, n_cheb_G the order N_G of ln G (0: N_G = N_Z)."""
    return dict(n_cheb=int(n_cheb), n_radial=int(n_radial), n_angular=int(n_angular),
                eps2=float(eps2), lambda2=float(lambda2), g2nc=float(g2nc), x_G=float(x_G),
                ginv_G=float(ginv_G), x_Z=float(lambda2 if x_Z is None else x_Z), zinv_Z=float(zinv_Z),
                kappa=float(kappa), delta=float(delta), radial_mode=int(radial_mode),
                extrap_mode=int(extrap_mode), precision=int(precision), n_cheb_G=int(n_cheb_G),
                angular_mode=int(angular_mode))


def workload_problem(name: str, **over) -> dict:
    kw = dict(WORKLOADS[name])
    kw.update(over)
    return problem(**kw)


def starting_guess(params: dict, seed: int = 0, noise: float = 0.01) -> np.ndarray:
    """Coefficients (a; b) of a smooth IR-power-law / UV-logarithm guess plus
    noise * N(0,1)/(j+1) drawn from numpy's default_rng(seed).

    The guess functions are  ln G0 = -kappa ln(x/(1+x)) + delta ln(1 + w ln(1+x))
    (for G(x_G)^{-1} = ginv_G > 0: ln G0 = -ln(ginv_G + (x/(1+x))^kappa) + the same
    UV term, so that G0 tends to 1/ginv_G in the infrared as the decoupling
    solutions do) and ln Z0 = 2 kappa ln(x/(1+x)) + gamma ln(1 + w ln(1+x)) + const with
    w = 11 g^2 N_c / (48 pi^2) and const fixing Z0(lambda2) = 1/zinv_Z; they are
    interpolated by numpy's Chebyshev routine in the variable
    s = ln(x / sqrt(eps2 lambda2)) / (ln(lambda2/eps2)/2) and converted to the
    b_0/2, a_0/2 convention of the expansion.
    """
    NZ = int(params["n_cheb"])
    NG = int(params.get("n_cheb_G", 0) or 0) or NZ
    kappa, delta = params["kappa"], params["delta"]
    gamma = -1.0 - 2.0 * delta
    w = 11.0 * params["g2nc"] / (48.0 * math.pi ** 2)
    l0 = 0.5 * math.log(params["eps2"] * params["lambda2"])
    l1 = 0.5 * math.log(params["lambda2"] / params["eps2"])

    ginv = float(params.get("ginv_G", 0.0))

    def lnG0(s):
        x = np.exp(l0 + l1 * s)
        uv = delta * np.log1p(w * np.log1p(x))
        if ginv > 0.0:
            # decoupling-type boundary value: G0 -> 1/ginv_G in the infrared
            return -np.log(ginv + (x / (1 + x)) ** kappa) + uv
        return -kappa * np.log(x / (1 + x)) + uv

    def lnZ0_raw(s):
        x = np.exp(l0 + l1 * s)
        return 2 * kappa * np.log(x / (1 + x)) + gamma * np.log1p(w * np.log1p(x))

    zs = -math.log(params["zinv_Z"]) - float(lnZ0_raw(np.array([1.0]))[0])
    cb = np.polynomial.chebyshev.chebinterpolate(lnG0, NG - 1)
    ca = np.polynomial.chebyshev.chebinterpolate(lambda s: lnZ0_raw(s) + zs, NZ - 1)
    cb = np.asarray(cb, dtype=np.float64); ca = np.asarray(ca, dtype=np.float64)
    cb[0] *= 2.0
    ca[0] *= 2.0
    rng = np.random.default_rng(seed)
    ca = ca + noise * rng.standard_normal(NZ) / (np.arange(NZ) + 1)
    cb = cb + noise * rng.standard_normal(NG) / (np.arange(NG) + 1)
    return np.concatenate([ca, cb]).astype(np.float64)


def schwinger_times(n_t: int = 4096, seed: int = 0, lo: float = 0.1, hi: float = 50.0) -> np.ndarray:
    """Euclidean times t ~ U[lo, hi] from numpy's default_rng(seed)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=int(n_t)).astype(np.float64)


def loss_momenta(n: int = 64, seed: int = 0, lo: float = 1e-4, hi: float = 1e4) -> np.ndarray:
    """Momenta x = p^2 log-uniform in [lo, hi] from numpy's default_rng(seed)."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=int(n))).astype(np.float64)


def target_factors(n: int = 64, seed: int = 1, spread: float = 0.05) -> np.ndarray:
    """Factors 1 + spread * U(-1, 1) from numpy's default_rng(seed): targets are a
    converged Z(x) times these."""
    return (1.0 + spread * np.random.default_rng(seed).uniform(-1.0, 1.0, size=int(n))).astype(np.float64)


BATCH_ORDERS = (24, 32, 48, 64)
BATCH_QUADRATURES = ((128, 64), (256, 128))


def batch_problems(n: int = 256, seed: int = 0, ginv_lo: float = 1e-3, ginv_hi: float = 1e-1) -> list:
    """A sweep of independent problems: per problem, N_Z and N_G drawn from
    BATCH_ORDERS, (n_radial, n_angular) from BATCH_QUADRATURES and G(x_G)^{-1}
    log-uniform in [ginv_lo, ginv_hi], from numpy's default_rng(seed) in that
    order; all other parameters as in problem()."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(int(n)):
        nz = int(rng.choice(BATCH_ORDERS))
        ng = int(rng.choice(BATCH_ORDERS))
        nr, na = BATCH_QUADRATURES[int(rng.integers(len(BATCH_QUADRATURES)))]
        ginv = float(math.exp(rng.uniform(math.log(ginv_lo), math.log(ginv_hi))))
        out.append(problem(nz, nr, na, n_cheb_G=ng, ginv_G=ginv))
    return out
