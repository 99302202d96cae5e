"""Pins for the paper's own quadrature (arXiv:1206.1779 Sec. 2 and Sec. 3):
the tanh-sinh rule in xi = cos theta for the angular integral (angular_mode 1)
and the radial split int_0^Lambda^2 = int_0^eps2 + int_eps2^x + int_x^Lambda^2
(radial_mode 1, the first piece over [1e-6 eps2, eps2]).

Closed forms: the angular moments of sin^2 and sin^4, a near-singular integrand
with a known integral, the angular averages of the kernels M and Q and of the
ghost kernel, and -- with both variants -- the self-energies of constant dressing
functions, which the split rule reaches to ~1e-15 because no piece contains the
kink at y = x."""
import math

import numpy as np
import pytest

from test_oracle_jacobian import fd_jacobian
from test_oracle_selfenergy import closed_forms, const_coeffs


def test_tanh_sinh_closed_forms(oracle, inputs):
    p = inputs.problem(4, 8, 64, angular_mode=1)
    _, _, th, wt = oracle.quadrature(p)
    # theta = 2 atan(e^{-u}) ascends; the last nodes round to pi in double precision
    # (their weights are below 1e-30)
    assert np.all(np.diff(th) >= 0) and th[0] > 0 and th[-1] <= math.pi
    assert abs(wt.sum() - math.pi) < 1e-14
    s2 = np.sin(th) ** 2
    assert abs(np.sum(wt * s2) - math.pi / 2) < 1e-14
    assert abs(np.sum(wt * s2 * s2) - 3 * math.pi / 8) < 1e-14
    # near the end point: int_0^pi sin^2 / (a - cos) = pi (a - sqrt(a^2 - 1)),
    # a - cos = (a - 1) + 2 sin^2(theta/2) without cancellation
    for a, tol in ((1.0001, 1e-13), (1 + 1e-6, 1e-11)):
        exact = math.pi * (a - math.sqrt(a * a - 1))

        def rel(mode):
            _, _, t, w = oracle.quadrature(inputs.problem(4, 8, 128, angular_mode=mode))
            v = np.sum(w * np.sin(t) ** 2 / ((a - 1) + 2 * np.sin(0.5 * t) ** 2))
            return abs(v / exact - 1)
        assert rel(1) < tol
    # the Gauss-Legendre rule of the same size misses the sharper one by far more
    assert rel(0) > 1e-7


@pytest.mark.parametrize("x,y", [(1e-3, 1.0), (0.5, 1.0), (7.0, 1.0), (2e-6, 3e5)])
def test_tanh_sinh_kernel_averages(oracle, inputs, x, y):
    _, _, th, wt = oracle.quadrature(inputs.problem(4, 8, 256, angular_mode=1))
    M = np.empty(th.size); Q = np.empty(th.size); z = np.empty(th.size)
    for i in range(th.size):
        M[i], Q[i], z[i] = oracle.kernels(x, y, th[i])
    s2 = np.sin(th) ** 2
    aM, aQ = (2 / math.pi) * np.sum(wt * s2 * M), (2 / math.pi) * np.sum(wt * s2 * Q)
    w = x / y
    if w < 1:
        eM, eQ = 0.75 - w / 4, -0.75 - 25 * w / 4 + 7 * w * w / 8
    else:
        eM, eQ = 0.75 / w - 0.25 / w ** 2, -0.75 - 25 / (4 * w) + 7 / (8 * w * w)
    assert abs(aM - eM) < 1e-12 and abs(aQ - eQ) < 1e-11
    eG = (3 * math.pi / 8) / max(x, y) ** 2
    assert abs(np.sum(wt * s2 * s2 / z ** 2) / eG - 1) < 1e-11


@pytest.mark.parametrize("x", [0.0, 3e-4, 37.0, 2.5e5, 1e6])
def test_split_radial_rule_pieces(oracle, inputs, x):
    p = inputs.problem(4, 24, 8, radial_mode=1)
    y, W = oracle.radial_rule(p, x)
    nr = 24
    assert y.size == 3 * nr
    e2, l2 = p["eps2"], p["lambda2"]
    xs = min(max(x, e2), l2)
    for (lo, hi), sl in (((1e-6 * e2, e2), slice(0, nr)), ((e2, xs), slice(nr, 2 * nr)),
                         ((xs, l2), slice(2 * nr, 3 * nr))):
        if hi > lo:
            assert np.all((y[sl] > lo) & (y[sl] < hi))
            assert abs(W[sl].sum() / (hi - lo) - 1) < 1e-13
            assert abs(np.sum(W[sl] / y[sl]) / math.log(hi / lo) - 1) < 1e-13
        else:
            assert np.all(W[sl] == 0.0)


@pytest.mark.parametrize("G0,Z0", [(1.3, 0.7), (0.45, 2.2)])
@pytest.mark.parametrize("x", [0.0, 3e-4, 37.0, 2.5e5])
def test_self_energy_with_paper_quadrature_is_spectral(oracle, inputs, x, G0, Z0):
    # constant dressing continued as constants below eps2: the split rule integrates
    # [1e-6 eps2, lambda2] with no kink inside a piece
    p = inputs.problem(2, 32, 128, extrap_mode=1, radial_mode=1, angular_mode=1)
    c = const_coeffs(2, G0, Z0)
    PiG, PiZ = oracle.self_energy(p, c, x)
    eG, eZ = closed_forms(dict(p, eps2=1e-6 * p["eps2"]), x, G0, Z0)
    assert abs(PiG / eG - 1) < 1e-12
    if x > 0:
        assert abs(PiZ / eZ - 1) < 1e-12
    # the single-rule default misses the same integral by orders of magnitude more
    if 1e-6 < x < 1e6:
        q = inputs.problem(2, 96, 128, extrap_mode=1)
        PiG0, _ = oracle.self_energy(q, c, x)
        e0, _ = closed_forms(q, x, G0, Z0)
        assert abs(PiG0 / e0 - 1) > 1e-9


@pytest.mark.parametrize("case", [
    dict(n_cheb=4, n_radial=8, n_angular=12, radial_mode=1),
    dict(n_cheb=5, n_cheb_G=3, n_radial=6, n_angular=16, angular_mode=1, ginv_G=0.05),
    dict(n_cheb=3, n_radial=6, n_angular=10, radial_mode=1, angular_mode=1, x_G=2e-3, ginv_G=0.02),
])
def test_jacobian_with_paper_quadrature(oracle, inputs, case):
    p = inputs.problem(**case)
    c = inputs.starting_guess(p, seed=9)
    J, F = oracle.newton_matrix(p, c)
    Jfd = fd_jacobian(oracle, p, c)
    rowmax = np.abs(J).max(axis=1, keepdims=True)
    assert np.all(np.abs(J - Jfd) <= 1e-6 * np.abs(J) + 1e-7 * rowmax)


def test_newton_converges_with_paper_quadrature(oracle, inputs):
    p = inputs.problem(12, 32, 32, radial_mode=1, angular_mode=1)
    c, it, hist = oracle.solve(p, inputs.starting_guess(p, seed=0), tol=1e-10, max_iter=40)
    assert hist[-1][1] < 1e-10
