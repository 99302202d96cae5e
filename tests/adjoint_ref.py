"""Loss gradient through the implicit function c*(theta), F(c*, theta) = 0,
composed from oracle routines only (test infrastructure):

    L(c) = sum_m (Z(x_m) - t_m)^2,  dL/da_j = sum_m 2 (Z_m - t_m) Z_m phi_j(x_m),
    J(c*)^T lambda = dL/dc*,        dL/dtheta = -lambda^T dF/dtheta,

theta = (g^2 Nc, G(x_G)^{-1}, Z(x_Z)^{-1}) as in arXiv:1206.1779 Sec. 2.2."""
import numpy as np


def z_at(oracle, p, c, x):
    _, lZ = oracle.dressing(p, c, x)
    return np.exp(lZ)


def loss(oracle, p, c, x, t):
    return float(np.sum((z_at(oracle, p, c, x) - t) ** 2))


def loss_grad_c(oracle, p, c, x, t):
    N = p["n_cheb"]
    Z = z_at(oracle, p, c, x)
    phi = np.array([oracle.basis(p, xm) for xm in x])
    g = np.zeros(2 * N)
    g[:N] = phi.T @ (2.0 * (Z - t) * Z)
    return g


def implicit_grad(oracle, p, c, x, t):
    """(dL/dtheta (3), lambda, dL/dc) at a converged c."""
    g = loss_grad_c(oracle, p, c, x, t)
    J, _ = oracle.newton_matrix(p, c)
    lam = oracle.lu_solve(np.ascontiguousarray(J.T), g)
    dF = oracle.param_derivatives(p, c)
    return -lam @ dF, lam, g
