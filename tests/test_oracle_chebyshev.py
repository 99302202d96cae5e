"""Pins of the Chebyshev expansion, the mapping s(x), collocation points and the
IR/UV continuation of the dressing functions (arXiv:1206.1779 Sec. 2 asymptotics,
Sec. 3 expansion and mapping)."""
import math

import numpy as np
import pytest


@pytest.fixture
def prob(inputs):
    return inputs.problem(16, 32, 16)


def test_map_end_points(oracle, prob):
    assert abs(oracle.map_s(prob, prob["eps2"]) + 1) < 1e-15
    assert abs(oracle.map_s(prob, prob["lambda2"]) - 1) < 1e-15
    assert abs(oracle.map_s(prob, math.sqrt(prob["eps2"] * prob["lambda2"]))) < 1e-15
    # the paper's base-10 form of the map
    lam, eps = math.sqrt(prob["lambda2"]), math.sqrt(prob["eps2"])
    for x in [3e-5, 0.7, 420.0]:
        s10 = math.log10(x / (lam * eps)) / math.log10(lam / eps)
        assert abs(oracle.map_s(prob, x) - s10) < 1e-14


def test_collocation_points_are_roots_of_T_N(oracle, prob):
    x = oracle.collocation(prob)
    N = prob["n_cheb"]
    assert np.all(np.diff(x) > 0)
    s = np.array([oracle.map_s(prob, xi) for xi in x])
    assert np.max(np.abs(np.cos(N * np.arccos(s)))) < 1e-13


def test_basis_is_cos_j_arccos(oracle, prob):
    N = prob["n_cheb"]
    for x in [2e-6, 1e-3, 1.0, 5e4, 9.9e5]:
        phi = oracle.basis(prob, x)
        s = oracle.map_s(prob, x)
        ref = np.cos(np.arange(N) * math.acos(s))
        ref[0] = 0.5
        assert np.max(np.abs(phi - ref)) < 1e-13
    # clamped outside [eps2, lambda2]
    lo = oracle.basis(prob, 1e-9)
    hi = oracle.basis(prob, 1e9)
    ref_lo = np.array([0.5] + [(-1.0) ** j for j in range(1, N)])
    ref_hi = np.array([0.5] + [1.0] * (N - 1))
    assert np.array_equal(lo, ref_lo) and np.array_equal(hi, ref_hi)


def test_series_reproduces_polynomial(oracle, prob):
    # ln G = polynomial of degree N-1 in s: interpolation at the collocation
    # points (discrete cosine transform) must reproduce it exactly.
    N = prob["n_cheb"]
    rng = np.random.default_rng(3)
    poly = rng.standard_normal(N) / (1 + np.arange(N))
    xs = oracle.collocation(prob)
    si = np.array([oracle.map_s(prob, x) for x in xs])
    vals = np.polynomial.polynomial.polyval(si, poly)
    j = np.arange(N)
    T = np.cos(np.outer(j, np.arccos(si)))
    b = (2.0 / N) * T @ vals  # b_0/2 convention
    c = np.concatenate([np.zeros(N), b])
    xt = np.exp(np.linspace(math.log(prob["eps2"]), math.log(prob["lambda2"]), 37))
    lG, lZ = oracle.dressing(prob, c, xt)
    st = np.array([oracle.map_s(prob, x) for x in xt])
    assert np.max(np.abs(lG - np.polynomial.polynomial.polyval(st, poly))) < 1e-12
    assert np.max(np.abs(lZ)) == 0.0


def test_ir_uv_continuation(oracle, prob, inputs):
    N = prob["n_cheb"]
    c = inputs.starting_guess(prob, seed=1)
    e2, l2, kap, dlt = prob["eps2"], prob["lambda2"], prob["kappa"], prob["delta"]
    gam = -1 - 2 * dlt
    # continuity at both matching points
    for xm in [e2, l2]:
        lG, lZ = oracle.dressing(prob, c, [xm * (1 - 1e-12), xm, xm * (1 + 1e-12)])
        assert np.ptp(lG) < 1e-10 and np.ptp(lZ) < 1e-10
    # IR: Z = A x^{2 kappa}, G = B x^{-kappa}  (log-log slopes)
    x1, x2 = 1e-9, 1e-12
    lG, lZ = oracle.dressing(prob, c, [x1, x2])
    dl = math.log(x1) - math.log(x2)
    assert abs((lG[0] - lG[1]) / dl + kap) < 1e-12
    assert abs((lZ[0] - lZ[1]) / dl - 2 * kap) < 1e-12
    # UV: G ~ (ln x)^delta and Z ~ (ln x)^gamma asymptotically
    xa, xb = 1e250, 1e300
    lG, lZ = oracle.dressing(prob, c, [xa, xb])
    dll = math.log(math.log(xb)) - math.log(math.log(xa))
    assert abs((lG[1] - lG[0]) / dll - dlt) < 5e-2 * abs(dlt)
    assert abs((lZ[1] - lZ[0]) / dll - gam) < 5e-2 * abs(gam)


@pytest.mark.parametrize("extrap", [0, 1])
def test_derivative_closure(oracle, inputs, extrap):
    # d ln G(x)/d b_j = d ln Z(x)/d a_j = phi_j(clamp x) in every region
    prob = inputs.problem(6, 8, 8, extrap_mode=extrap)
    N = prob["n_cheb"]
    c = inputs.starting_guess(prob, seed=2)
    xs = np.array([1e-10, 3e-6, 0.5, 2e5, 3e7])
    for j in range(2 * N):
        h = 1e-6
        cp = c.copy(); cp[j] += h
        cm = c.copy(); cm[j] -= h
        gp, zp = oracle.dressing(prob, cp, xs)
        gm, zm = oracle.dressing(prob, cm, xs)
        dG = (gp - gm) / (2 * h)
        dZ = (zp - zm) / (2 * h)
        for m, x in enumerate(xs):
            phi = oracle.basis(prob, x)
            if j < N:
                assert abs(dZ[m] - phi[j]) < 1e-8 and abs(dG[m]) < 1e-8
            else:
                assert abs(dG[m] - phi[j - N]) < 1e-8 and abs(dZ[m]) < 1e-8
