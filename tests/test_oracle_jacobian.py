"""Pin of the oracle's analytic Newton matrix against central finite differences
of its residual (the paper's own Jacobian recipe, arXiv:1206.1779 Sec. 4.2,
Eq. (derivatives), with the step h_j = 1e-4 max(|c_j|, 1e-3); the paper used about 1e-5 a_j)."""
import numpy as np
import pytest


def fd_jacobian(oracle, p, c, rel=1e-4):
    n = c.size
    J = np.empty((n, n))
    for j in range(n):
        h = rel * max(abs(c[j]), 1e-3)
        cp = c.copy(); cp[j] += h
        cm = c.copy(); cm[j] -= h
        J[:, j] = (oracle.residual(p, cp) - oracle.residual(p, cm)) / (2 * h)
    return J


CASES = [
    dict(n_cheb=4, n_radial=16, n_angular=8),
    dict(n_cheb=5, n_radial=12, n_angular=6, ginv_G=0.05, x_G=2e-3, x_Z=3e4),
    dict(n_cheb=6, n_radial=20, n_angular=10, extrap_mode=1, zinv_Z=2.0),
    dict(n_cheb=3, n_radial=9, n_angular=5, eps2=1e-4, lambda2=1e3, x_Z=1e3),
]


@pytest.mark.parametrize("case", CASES)
def test_jacobian_matches_central_differences(oracle, inputs, case):
    p = inputs.problem(**case)
    c = inputs.starting_guess(p, seed=7)
    J, F = oracle.newton_matrix(p, c)
    assert np.allclose(F, oracle.residual(p, c), rtol=0, atol=0)
    Jfd = fd_jacobian(oracle, p, c)
    rowmax = np.abs(J).max(axis=1, keepdims=True)
    err = np.abs(J - Jfd)
    # FD truncation ~h^2 and cancellation noise ~eps*|Pi|/h set the bound
    assert np.all(err <= 1e-6 * np.abs(J) + 1e-7 * rowmax), err.max()


def test_block_layout(oracle, inputs):
    # rows (z(x_0..); g(x_0..)), columns (a; b): the z-rows see b only through
    # the vertex model and the ghost loop, the g-rows see a only through Z(z);
    # the diagonal-type terms -Z^{-1} phi_j(x_i), -G^{-1} phi_j(x_i) sit in the
    # (z,a) and (g,b) blocks.
    p = inputs.problem(4, 10, 6)
    c = inputs.starting_guess(p, seed=1)
    J, _ = oracle.newton_matrix(p, c)
    N = 4
    # perturbing a by a constant shift of ln Z (a_0 -> a_0 + 2 t) changes Z^{-1}(x_i)
    # by -t Z^{-1} at first order: column 0 of the (z,a) block carries -Z^{-1}/2 + ...
    x = oracle.collocation(p)
    lG, lZ = oracle.dressing(p, c, x)
    dZ = oracle.self_energy(p, c, x[0], grad=True)[3]
    dZref = oracle.self_energy(p, c, p["x_Z"], grad=True)[3]
    assert abs(J[0, 0] - (-np.exp(-lZ[0]) * 0.5 - dZ[0] + dZref[0])) < 1e-12 * np.abs(J[0]).max()
    dG = oracle.self_energy(p, c, x[1], grad=True)[2]
    dGref = oracle.self_energy(p, c, p["x_G"], grad=True)[2]
    assert abs(J[N + 1, N + 2] - (-np.exp(-lG[1]) * oracle.basis(p, x[1])[2] - dG[N + 2] + dGref[N + 2])) \
        < 1e-12 * np.abs(J[N + 1]).max()


def test_magnitude_sums_bound_entries(oracle, inputs):
    # A_ij (sum of |summands|) >= |J_ij| and AF_i >= |F_i|, with equality for
    # entries whose summands share one sign; scaling c by nothing changes A
    for case in CASES[:2]:
        p = inputs.problem(**case)
        c = inputs.starting_guess(p, seed=7)
        J, F = oracle.newton_matrix(p, c)
        A, AF = oracle.newton_matrix_magnitudes(p, c)
        assert np.all(A >= np.abs(J) * (1 - 1e-14))
        assert np.all(AF >= np.abs(F) * (1 - 1e-14))
        assert np.all(np.isfinite(A)) and np.all(A > 0)
