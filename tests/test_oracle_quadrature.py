"""Pins of the oracle's quadrature rules (radial Gauss-Legendre in ln y, angular
Gauss-Legendre in theta; arXiv:1206.1779 Sec. 2, O(4) reduction and radial rule)."""
import math

import numpy as np
import pytest


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 16, 31, 64, 128, 257])
def test_gauss_legendre_exact_for_polynomials(oracle, n):
    x, w = oracle.gauss_legendre(n)
    assert np.all(np.diff(x) > 0)
    for k in range(0, 2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        got = float(np.sum(w * x ** k))
        assert abs(got - exact) <= 4e-15 * max(1.0, n / 8), (n, k, got, exact)


@pytest.mark.parametrize("n", [4, 32, 100])
def test_gauss_legendre_matches_numpy(oracle, n):
    x, w = oracle.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.max(np.abs(x - xr)) < 1e-15
    # numpy's own weights carry ~1e-12 relative error at n = 100
    assert np.max(np.abs(w - wr) / wr) < 5e-11
    assert np.max(np.abs(x + x[::-1])) < 1e-15


def test_gauss_legendre_against_40_digit_roots(oracle):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    n = 100
    x, w = oracle.gauss_legendre(n)
    for i in [0, 7, 49]:
        r = mp.findroot(lambda t: mp.legendre(n, t), mp.mpf(x[i]))
        dp = mp.diff(lambda t: mp.legendre(n, t), r)
        we = 2 / ((1 - r ** 2) * dp ** 2)
        assert abs(x[i] - float(r)) < 2e-16
        assert abs(w[i] / float(we) - 1) < 1e-12


def test_gauss_legendre_large_n_weights(oracle):
    x, w = oracle.gauss_legendre(8192)
    assert abs(w.sum() - 2.0) < 1e-13
    assert abs(np.sum(w * x * x) - 2.0 / 3.0) < 1e-13


def test_radial_rule_closed_forms(oracle, inputs):
    p = inputs.problem(8, 64, 32)
    y, W, th, wt = oracle.quadrature(p)
    e2, l2 = p["eps2"], p["lambda2"]
    assert np.all(np.diff(y) > 0) and y[0] > e2 and y[-1] < l2
    # int dy = L^2 - e^2 ;  int dy / y = ln(L^2/e^2) ;  int dy / y^2 = 1/e^2 - 1/L^2
    assert abs(W.sum() / (l2 - e2) - 1) < 1e-13
    assert abs(np.sum(W / y) / math.log(l2 / e2) - 1) < 1e-14
    assert abs(np.sum(W / y ** 2) / (1 / e2 - 1 / l2) - 1) < 1e-13


def test_angular_rule_closed_forms(oracle, inputs):
    p = inputs.problem(8, 16, 32)
    _, _, th, wt = oracle.quadrature(p)
    assert np.all((th > 0) & (th < math.pi))
    assert abs(wt.sum() - math.pi) < 1e-14
    # 4-d measure: int sin^2 = pi/2 ; ghost measure int sin^4 = 3 pi / 8
    assert abs(np.sum(wt * np.sin(th) ** 2) - math.pi / 2) < 1e-14
    assert abs(np.sum(wt * np.sin(th) ** 4) - 3 * math.pi / 8) < 1e-14
