"""Pins for separate Chebyshev orders N_Z (ln Z) and N_G (ln G): the gluon rows of
the residual sit at the N_Z mapped roots, the ghost rows at the N_G roots
(arXiv:1206.1779 Sec. 3 with one expansion per dressing function).

- A dressing function does not depend on how many zero coefficients pad its
  expansion, so self-energies and their coefficient derivatives computed with
  N_G = 5 equal those with N_G = 8 and b_5 = b_6 = b_7 = 0.
- The residual rows are the defining formulas at the right points, rebuilt here
  from self_energy and dressing.
- The Newton matrix matches central differences of the residual.
- Newton converges for N_Z != N_G."""
import numpy as np
import pytest

from test_oracle_jacobian import fd_jacobian


def pad_b(c, nz, ng, ng_big):
    return np.concatenate([c[:nz], c[nz:nz + ng], np.zeros(ng_big - ng)])


@pytest.mark.parametrize("nz,ng", [(6, 4), (4, 7)])
def test_padding_invariance_of_self_energy(oracle, inputs, nz, ng):
    small = inputs.problem(nz, 14, 10, n_cheb_G=ng)
    big = inputs.problem(nz, 14, 10, n_cheb_G=ng + 3)
    c = inputs.starting_guess(small, seed=2)
    assert c.size == nz + ng
    cb = pad_b(c, nz, ng, ng + 3)
    for x in (0.0, 3e-4, 0.7, 2e3):
        a = oracle.self_energy(small, c, x, grad=True)
        b = oracle.self_energy(big, cb, x, grad=True)
        assert a[0] == pytest.approx(b[0], rel=1e-14, abs=1e-300)
        assert a[1] == pytest.approx(b[1], rel=1e-14, abs=1e-300)
        for da, db in ((a[2], b[2]), (a[3], b[3])):
            assert da.size == nz + ng and db.size == nz + ng + 3
            scale = np.abs(db).max() + 1e-300
            assert np.allclose(da, db[:nz + ng], rtol=0, atol=1e-14 * scale)


@pytest.mark.parametrize("nz,ng", [(6, 4), (4, 7)])
def test_residual_rows_at_their_points(oracle, inputs, nz, ng):
    p = inputs.problem(nz, 12, 8, n_cheb_G=ng, ginv_G=0.02)
    c = inputs.starting_guess(p, seed=3)
    F = oracle.residual(p, c)
    assert F.size == nz + ng
    xz, xg = oracle.collocation(p), oracle.collocation(p, ghost=True)
    assert xz.size == nz and xg.size == ng
    _, piz_ref = oracle.self_energy(p, c, p["x_Z"])
    pig_ref, _ = oracle.self_energy(p, c, p["x_G"])
    _, lZ = oracle.dressing(p, c, xz)
    lG, _ = oracle.dressing(p, c, xg)
    for i in range(nz):
        _, piz = oracle.self_energy(p, c, xz[i])
        expect = np.exp(-lZ[i]) - p["zinv_Z"] - piz + piz_ref
        assert F[i] == pytest.approx(expect, rel=1e-13, abs=1e-13 * abs(piz))
    for i in range(ng):
        pig, _ = oracle.self_energy(p, c, xg[i])
        expect = np.exp(-lG[i]) - p["ginv_G"] - pig + pig_ref
        assert F[nz + i] == pytest.approx(expect, rel=1e-13, abs=1e-13 * abs(pig))


@pytest.mark.parametrize("case", [
    dict(n_cheb=5, n_cheb_G=3, n_radial=12, n_angular=6),
    dict(n_cheb=3, n_cheb_G=6, n_radial=16, n_angular=8, ginv_G=0.05, x_G=2e-3, x_Z=3e4),
])
def test_jacobian_matches_central_differences_separate_orders(oracle, inputs, case):
    p = inputs.problem(**case)
    c = inputs.starting_guess(p, seed=7)
    J, F = oracle.newton_matrix(p, c)
    n = case["n_cheb"] + case["n_cheb_G"]
    assert J.shape == (n, n)
    Jfd = fd_jacobian(oracle, p, c)
    rowmax = np.abs(J).max(axis=1, keepdims=True)
    assert np.all(np.abs(J - Jfd) <= 1e-6 * np.abs(J) + 1e-7 * rowmax)
    # the -Z^{-1} phi_j block stops at column N_Z, the -G^{-1} phi_j block starts there
    A, _ = oracle.newton_matrix_magnitudes(p, c)
    assert A.shape == (n, n)


def test_newton_converges_with_separate_orders(oracle, inputs):
    p = inputs.problem(12, 48, 24, n_cheb_G=8)
    c, it, hist = oracle.solve(p, inputs.starting_guess(p, seed=0), tol=1e-10, max_iter=40)
    assert hist[-1][1] < 1e-10
    assert c.size == 20
