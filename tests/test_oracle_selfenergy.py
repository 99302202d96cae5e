"""Pins of the ghost and gluon self-energies (arXiv:1206.1779 Sec. 2: ghost and
gluon equations, O(4) measure, three-gluon vertex model, MOM residuals of Sec. 3)
against closed-form integrals for constant dressing functions."""
import math

import numpy as np
import pytest


def const_coeffs(N, G0, Z0):
    c = np.zeros(2 * N)
    c[0] = 2 * math.log(Z0)      # a_0 / 2 = ln Z0
    c[N] = 2 * math.log(G0)      # b_0 / 2 = ln G0
    return c


def closed_forms(p, x, G0, Z0):
    """Exact Pi_G(x), Pi_Z(x) on [eps2, lambda2] for G = G0, Z = Z0 everywhere."""
    e2, l2 = p["eps2"], p["lambda2"]
    K = p["g2nc"] / (2 * math.pi) ** 3
    dl = p["delta"]
    pG, qZ = -2 - 6 * dl, -3 * dl
    W0 = G0 ** (2 * pG) * Z0 ** (2 * qZ)
    # ghost: int dy y (3 pi/8)/max(x,y)^2
    A, B = e2, min(max(x, e2), l2)
    C, D = max(x, e2), l2
    ig = (B * B - A * A) / (2 * x * x) if x > 0 else 0.0
    ig += math.log(D / C) if C < D else 0.0
    PiG = -K * G0 * Z0 * (3 * math.pi / 8) * ig
    if x == 0:
        return PiG, None
    IM = (3 / (8 * x)) * (B * B - A * A) - (B ** 3 - A ** 3) / (12 * x * x)
    IQ = -0.75 * (B - A) - (25 / (8 * x)) * (B * B - A * A) + (7 / (24 * x * x)) * (B ** 3 - A ** 3)
    if C < D:
        IM += 0.75 * (D - C) - (x / 4) * math.log(D / C)
        IQ += -0.75 * (D - C) - (25 * x / 4) * math.log(D / C) + (7 * x * x / 8) * (1 / C - 1 / D)
    PiZ = (K / (3 * x)) * (math.pi / 2) * (W0 * IQ + G0 * G0 * IM)
    return PiG, PiZ


@pytest.mark.parametrize("G0,Z0", [(1.0, 1.0), (1.3, 0.7), (0.45, 2.2)])
@pytest.mark.parametrize("x", [0.0, 1e-7, 4e6])
def test_self_energy_outside_range_spectral(oracle, inputs, x, G0, Z0):
    # x outside [eps2, lambda2]: the y-integrand has no kink, Gauss-Legendre is spectral
    p = inputs.problem(3, 160, 96, extrap_mode=1)
    c = const_coeffs(3, G0, Z0)
    PiG, PiZ = oracle.self_energy(p, c, x)
    eG, eZ = closed_forms(p, x, G0, Z0)
    assert abs(PiG / eG - 1) < 1e-12
    if x > 0:
        # the Q and M terms cancel their quadratic (lambda2/x) parts when
        # W0 = G0^2; bound the rounding by the size of the cancelled terms
        K = p["g2nc"] / (2 * math.pi) ** 3
        W0 = G0 ** (2 * (-2 - 6 * p["delta"])) * Z0 ** (2 * (-3 * p["delta"]))
        S = K / (3 * x) * (math.pi / 2) * (W0 + G0 * G0) * p["lambda2"]
        assert abs(PiZ - eZ) <= 1e-12 * abs(eZ) + 1e-14 * S
    else:
        assert PiZ == 0.0


@pytest.mark.parametrize("x", [3e-4, 37.0, 2.5e5])
def test_self_energy_inside_range(oracle, inputs, x):
    # inside the range the single log-y rule sees the kink at y = x (reading of
    # the radial split): it converges algebraically, so the bound is loose
    G0, Z0 = 1.3, 0.7
    p = inputs.problem(2, 3000, 256, extrap_mode=1)
    c = const_coeffs(2, G0, Z0)
    PiG, PiZ = oracle.self_energy(p, c, x)
    eG, eZ = closed_forms(p, x, G0, Z0)
    assert abs(PiG / eG - 1) < 1e-5
    assert abs(PiZ / eZ - 1) < 1e-4


def test_closed_forms_carry_one_loop_logs(inputs):
    # the closed forms used above must reproduce the one-loop coefficients of
    # d Pi / d ln x for eps2 << x << lambda2 with G = Z = 1:
    # (g^2 Nc / 16 pi^2) * 3/4 (ghost) and * 13/6 (gluon)
    p = inputs.problem(2, 8, 8, eps2=1e-6, lambda2=1e6, x_Z=1e6)
    a = p["g2nc"] / (16 * math.pi ** 2)
    h = 1e-2
    gp, zp = closed_forms(p, math.exp(h), 1.0, 1.0)
    gm, zm = closed_forms(p, math.exp(-h), 1.0, 1.0)
    assert abs((gp - gm) / (2 * h) / (0.75 * a) - 1) < 1e-4
    assert abs((zp - zm) / (2 * h) / (13.0 / 6.0 * a) - 1) < 1e-4


def test_residual_structure(oracle, inputs):
    # F rows: Z(x_i)^{-1} - Z(x_Z)^{-1} - Pi_Z(x_i) + Pi_Z(x_Z), then the ghost rows
    p = inputs.problem(5, 24, 16, ginv_G=0.03, zinv_Z=3.1)
    c = inputs.starting_guess(p, seed=4)
    F = oracle.residual(p, c)
    x = oracle.collocation(p)
    lG, lZ = oracle.dressing(p, c, x)
    gZ = oracle.self_energy(p, c, p["x_Z"])
    gG = oracle.self_energy(p, c, p["x_G"])
    N = p["n_cheb"]
    for i in range(N):
        PiG, PiZ = oracle.self_energy(p, c, x[i])
        fz = math.exp(-lZ[i]) - p["zinv_Z"] - PiZ + gZ[1]
        fg = math.exp(-lG[i]) - p["ginv_G"] - PiG + gG[0]
        assert abs(F[i] - fz) <= 1e-14 * (abs(PiZ) + abs(gZ[1]) + math.exp(-lZ[i]))
        assert abs(F[N + i] - fg) <= 1e-14 * (abs(PiG) + abs(gG[0]) + math.exp(-lG[i]))
