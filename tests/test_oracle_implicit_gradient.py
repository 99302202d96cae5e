"""Pin of the implicit-function gradient composed from oracle routines
(tests/adjoint_ref.py): dL/dtheta = -lambda^T dF/dtheta with J^T lambda = dL/dc
at the converged coefficients, against central differences of the loss over
converged solves at theta +- h (h = 1e-6 relative), for the decoupling-type
boundary value G(x_G)^{-1} = 0.01 (arXiv:1206.1779 Sec. 2.1)."""
import numpy as np
import pytest

import adjoint_ref as R


def converge(oracle, p, c, n_relax=8, rho=0.5, tol=1e-11, max_iter=60):
    for it in range(max_iter):
        c_new, st = oracle.newton_step(p, c, rho if it < n_relax else 1.0)
        if st[1] < tol:
            return c
        c = c_new
    raise AssertionError("oracle solve did not converge")


@pytest.fixture(scope="module")
def converged(oracle, inputs):
    p = inputs.problem(n_cheb=8, n_radial=32, n_angular=16, ginv_G=0.01)
    c = converge(oracle, p, inputs.starting_guess(p, seed=0))
    x = inputs.loss_momenta(16)
    t = R.z_at(oracle, p, c, x) * inputs.target_factors(16)
    return p, c, x, t


@pytest.mark.parametrize("name,col", [("g2nc", 0), ("ginv_G", 1), ("zinv_Z", 2)])
def test_implicit_gradient_matches_central_differences(oracle, converged, name, col):
    p, c, x, t = converged
    grad, lam, g = R.implicit_grad(oracle, p, c, x, t)
    h = 1e-6 * abs(p[name])
    L = []
    for sgn in (1.0, -1.0):
        pp = dict(p)
        pp[name] += sgn * h
        L.append(R.loss(oracle, pp, converge(oracle, pp, c, n_relax=0), x, t))
    fd = (L[0] - L[1]) / (2 * h)
    # FD truncation ~1e-12 relative; the solves stop at a dimensionless residual
    # of 1e-11, which moves the quotient by up to a few 1e-6 relative
    assert abs(fd - grad[col]) <= 5e-5 * abs(grad[col]), (name, fd, grad[col])


def test_adjoint_solves_transposed_system(oracle, converged):
    p, c, x, t = converged
    grad, lam, g = R.implicit_grad(oracle, p, c, x, t)
    J, _ = oracle.newton_matrix(p, c)
    assert np.allclose(J.T @ lam, g, rtol=0, atol=1e-10 * np.abs(g).max())
    # the gradient in c is non-zero in the Z block only (the loss reads Z)
    N = p["n_cheb"]
    assert np.all(g[N:] == 0.0) and np.abs(g[:N]).max() > 0
