"""Pins of the gluon-equation kernels M and Q (arXiv:1206.1779 Sec. 2, kernel
equations with the +15/4 term) and of the ghost angular integral.

The oracle evaluates M = y sin^2(theta)/z and Q = quartic(sin^2(theta/2))/(2 z^2),
cancellation-free forms derived from the printed ones.  They are pinned against
the printed forms in 60-digit arithmetic and against closed-form angular
averages of the 4-d measure."""
import json
import math
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def printed_kernels(mp, x, y, th):
    """M and Q exactly as printed in Sec. 2 (with the 15/4 of the footnote)."""
    x, y, th = mp.mpf(x), mp.mpf(y), mp.mpf(th)
    z = x + y - 2 * mp.sqrt(x * y) * mp.cos(th)
    M = (1 / z) * (-x / 4 + y / 2 - y * y / (4 * x)) + mp.mpf(1) / 2 + y / (2 * x) - z / (4 * x)
    c15 = mp.mpf(json.load(open(GOLD))["quadratic_divergence_term"]["value"])
    Q = ((1 / z ** 2) * (x ** 3 / (8 * y) + x ** 2 - mp.mpf(9) / 4 * x * y + y ** 2 + y ** 3 / (8 * x))
         + (1 / z) * (x ** 2 / y - 4 * (x + y) + y ** 2 / x) - (mp.mpf(9) / 4 * x / y + 4 + mp.mpf(9) / 4 * y / x)
         + z * (1 / x + 1 / y) + z ** 2 / (8 * x * y) + c15)
    return M, Q, z


def test_kernels_equal_printed_forms(oracle):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    rng = np.random.default_rng(11)
    for _ in range(300):
        x = 10.0 ** rng.uniform(-6, 6)
        y = 10.0 ** rng.uniform(-6, 6)
        th = rng.uniform(1e-3, math.pi - 1e-3)
        M, Q, z = oracle.kernels(x, y, th)
        Me, Qe, ze = printed_kernels(mp, x, y, th)
        assert abs(z - float(ze)) <= 2e-15 * abs(float(ze))
        assert abs(M - float(Me)) <= 1e-14 * abs(float(Me))
        # Q can pass through zero in theta: compare on the scale of its terms
        scale = abs(float(Qe)) + 1.0
        assert abs(Q - float(Qe)) <= 1e-13 * scale, (x, y, th, Q, float(Qe))


def _angular_avg(oracle, x, y, n=400, weight=2):
    th, wt = np.polynomial.legendre.leggauss(n)
    th = 0.5 * math.pi * (1 + th)
    wt = 0.5 * math.pi * wt
    M = np.empty(n); Q = np.empty(n); z = np.empty(n)
    for i in range(n):
        M[i], Q[i], z[i] = oracle.kernels(x, y, th[i])
    s2 = np.sin(th) ** 2
    return (2 / math.pi) * np.sum(wt * s2 * M), (2 / math.pi) * np.sum(wt * s2 * Q), np.sum(wt * s2 * s2 / z ** 2)


@pytest.mark.parametrize("x,y", [(1e-3, 1.0), (0.1, 1.0), (0.5, 1.0), (1.0, 0.5), (7.0, 1.0),
                                 (1e3, 1.0), (2e-6, 3e5), (4e5, 1e-6)])
def test_angular_averages_closed_form(oracle, x, y):
    aM, aQ, gh = _angular_avg(oracle, x, y)
    w = x / y
    if w < 1:
        eM, eQ = 0.75 - w / 4, -0.75 - 25 * w / 4 + 7 * w * w / 8
    else:
        eM, eQ = 0.75 / w - 0.25 / w ** 2, -0.75 - 25 / (4 * w) + 7 / (8 * w * w)
    assert abs(aM - eM) < 1e-12
    assert abs(aQ - eQ) < 1e-11
    # ghost: int_0^pi sin^4 / z^2 dtheta = (3 pi / 8) / max(x, y)^2
    eG = (3 * math.pi / 8) / max(x, y) ** 2
    assert abs(gh / eG - 1) < 1e-11


def test_quadratic_divergence_cancels(oracle):
    # y >> x: <M> -> 3/4 and <Q> -> -3/4 (the 15/4 makes them cancel)
    aM, aQ, _ = _angular_avg(oracle, 1e-4, 1e4)
    assert abs(aM - 0.75) < 1e-7 and abs(aQ + 0.75) < 1e-6


def test_Q_symmetric(oracle):
    rng = np.random.default_rng(5)
    for _ in range(50):
        x, y = 10.0 ** rng.uniform(-4, 4, size=2)
        th = rng.uniform(0, math.pi)
        _, q1, _ = oracle.kernels(x, y, th)
        _, q2, _ = oracle.kernels(y, x, th)
        assert abs(q1 - q2) <= 1e-13 * (abs(q1) + 1)
