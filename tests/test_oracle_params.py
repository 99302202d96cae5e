"""Pin of the oracle's parameter derivatives dF/d(g^2 Nc, G(x_G)^{-1}, Z(x_Z)^{-1}).

The coupling enters the renormalised equations (arXiv:1206.1779 Sec. 2, Eqs. for
Pi_G and Pi_Z with the MOM subtraction of Sec. 2.2) through the prefactor
g^2 Nc/(2 pi)^3 and through omega = 11 g^2 Nc/(48 pi^2) of the UV forms of G and
Z (Sec. 3.1).  The two boundary values enter linearly with coefficient -1.  The
pins are central differences of the oracle residual in each parameter, exact
differences for the linear ones, and a check that dropping the omega term
fails the difference test."""
import numpy as np
import pytest

CASES = [
    dict(n_cheb=4, n_radial=16, n_angular=8),
    dict(n_cheb=5, n_radial=12, n_angular=6, ginv_G=0.05, x_G=2e-3, x_Z=3e4),
    dict(n_cheb=6, n_radial=20, n_angular=10, extrap_mode=1, zinv_Z=2.0),
    dict(n_cheb=3, n_radial=9, n_angular=5, eps2=1e-4, lambda2=1e3, x_Z=1e3),
]


def central_difference(oracle, p, c, name, h):
    pp = dict(p); pp[name] += h
    pm = dict(p); pm[name] -= h
    return (oracle.residual(pp, c) - oracle.residual(pm, c)) / (2 * h)


@pytest.mark.parametrize("case", CASES)
def test_coupling_derivative_matches_central_differences(oracle, inputs, case):
    p = inputs.problem(**case)
    c = inputs.starting_guess(p, seed=3)
    dF = oracle.param_derivatives(p, c)
    assert dF.shape == (2 * p["n_cheb"], 3)
    fd = central_difference(oracle, p, c, "g2nc", 1e-5 * p["g2nc"])
    scale = np.abs(dF[:, 0]).max()
    # truncation ~h^2 relative, cancellation ~eps |F| / h per entry
    assert np.all(np.abs(fd - dF[:, 0]) <= 1e-7 * np.abs(dF[:, 0]) + 1e-12 * scale)


@pytest.mark.parametrize("case", CASES)
def test_boundary_values_enter_linearly(oracle, inputs, case):
    p = inputs.problem(**case)
    N = p["n_cheb"]
    c = inputs.starting_guess(p, seed=4)
    dF = oracle.param_derivatives(p, c)
    F = oracle.residual(p, c)
    for name, col, rows in (("zinv_Z", 2, slice(0, N)), ("ginv_G", 1, slice(N, 2 * N))):
        expect = np.zeros(2 * N)
        expect[rows] = -1.0
        assert np.array_equal(dF[:, col], expect)
        pp = dict(p); pp[name] += 0.5
        diff = oracle.residual(pp, c) - F
        assert np.allclose(diff, 0.5 * expect, rtol=0, atol=4 * np.finfo(float).eps * np.abs(F).max())


def test_omega_term_is_needed(oracle, inputs):
    # With the UV form active (extrap_mode 0, z above lambda2 inside the angular
    # integral), Pi/g2nc alone misses the omega term by far more than the FD noise.
    p = inputs.problem(n_cheb=5, n_radial=16, n_angular=10)
    N = p["n_cheb"]
    c = inputs.starting_guess(p, seed=5)
    F = oracle.residual(p, c)
    x = oracle.collocation(p)
    lG, lZ = oracle.dressing(p, c, x)
    naive = np.empty(2 * N)
    # F_z = Z^{-1} - zinv - (Pi_Z(x_i) - Pi_Z(x_Z)), and Pi is proportional to K
    naive[:N] = (F[:N] - np.exp(-lZ) + p["zinv_Z"]) / p["g2nc"]
    naive[N:] = (F[N:] - np.exp(-lG) + p["ginv_G"]) / p["g2nc"]
    fd = central_difference(oracle, p, c, "g2nc", 1e-5 * p["g2nc"])
    dF = oracle.param_derivatives(p, c)[:, 0]
    scale = np.abs(dF).max()
    assert np.all(np.abs(fd - dF) <= 1e-7 * np.abs(dF) + 1e-12 * scale)
    # the UV rows differ from Pi/g2nc at the per-mille level and beyond
    assert np.max(np.abs(fd - naive) / np.abs(fd)) >= 1e-3
