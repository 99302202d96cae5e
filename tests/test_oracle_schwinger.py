"""Pins of the oracle's Schwinger function (arXiv:1206.1779 Sec. 2.2,
Delta(t) = (1/pi) int_0^inf d|p| cos(t|p|) sigma(p^2), sigma = Z/p^2) and of its
mapped Gauss-Legendre rule (Sec. 5)."""
import math

import numpy as np
import pytest


def test_nodes_integrate_known_functions(oracle, inputs):
    p = inputs.problem(4, 8, 8, eps2=1e-6, lambda2=1e4, x_Z=1e4)
    pn, wn = oracle.schwinger_nodes(p, 512)
    eps, lam = 1e-3, 100.0
    assert np.all(np.diff(pn) > 0) and pn[0] > eps and pn[-1] < lam
    assert abs(np.sum(wn) / (lam - eps) - 1) < 1e-13
    assert abs(np.sum(wn / (1 + pn ** 2)) - (math.atan(lam) - math.atan(eps))) < 1e-13


def massive_coefficients(p, m2):
    """a-coefficients of ln Z for Z(x) = x/(x+m2), so sigma = 1/(p^2 + m2)."""
    N = p["n_cheb"]
    l0 = 0.5 * math.log(p["eps2"] * p["lambda2"])
    l1 = 0.5 * math.log(p["lambda2"] / p["eps2"])

    def lnZ(s):
        x = np.exp(l0 + l1 * s)
        return np.log(x) - np.log(x + m2)

    a = np.asarray(np.polynomial.chebyshev.chebinterpolate(lnZ, N - 1), dtype=np.float64)
    a[0] *= 2
    return np.concatenate([a, np.zeros(N)])


@pytest.mark.parametrize("t", [0.3, 1.0, 2.5, 5.0])
def test_schwinger_of_massive_propagator(oracle, inputs, t):
    integrate = pytest.importorskip("scipy.integrate")
    m = 1.0
    p = inputs.problem(128, 8, 8, eps2=1e-6, lambda2=1e4, x_Z=1e4)
    c = massive_coefficients(p, m * m)
    got = oracle.schwinger(p, c, np.array([t]), 8192)[0]
    eps, lam = 1e-3, 100.0
    f = lambda q: 1.0 / (q * q + m * m)
    trunc = integrate.quad(f, eps, lam, weight="cos", wvar=t, epsabs=1e-14, epsrel=1e-13, limit=400)[0] / math.pi
    assert abs(got - trunc) < 1e-9
    # the full-line transform is exp(-m t)/(2m); the tails account for the rest
    lo = integrate.quad(f, 0.0, eps, weight="cos", wvar=t, epsabs=1e-15)[0]
    hi = integrate.quad(f, lam, np.inf, weight="cos", wvar=t, epsabs=1e-15)[0]
    assert abs(trunc + (lo + hi) / math.pi - math.exp(-m * t) / (2 * m)) < 1e-10


def test_schwinger_linear_in_sigma(oracle, inputs):
    # Delta is linear in sigma = Z/p^2: doubling Z (a_0 += 2 ln 2) doubles Delta
    p = inputs.problem(16, 8, 8)
    c = inputs.starting_guess(p, seed=0)
    t = inputs.schwinger_times(16, seed=3)
    d1 = oracle.schwinger(p, c, t, 1024)
    c2 = c.copy(); c2[0] += 2 * math.log(2.0)
    d2 = oracle.schwinger(p, c2, t, 1024)
    assert np.allclose(d2, 2 * d1, rtol=1e-12, atol=1e-15)
