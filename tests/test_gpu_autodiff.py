"""GPU parity of the differentiation entry points (dse_vjp, dse_param_derivatives,
dse_adjoint_solve, dse_dressing_vjp, dse_plan_set_couplings) and of the
torch.autograd Functions built on them, against the FP64 oracle
(arXiv:1206.1779 Sec. 2-3; the derivative closure of Sec. 3 and the coupling
dependence of the Sec. 2 UV forms).

Bars, per entry, from the Newton-matrix bar of tests/gpu_util.py
(bar_ij = 1e-11 |J_ij| + (1e-13 + 16 j^2 u) A_ij):
  v^T J:          sum_i |v_i| bar_ij + 4 (2N) u sum_i |v_i J_ij|
  dF/dg2nc:       1e-11 |o| + 1e-12 AF_i / g2nc   (AF: magnitude sum of F_i; the
                  omega term is bounded by a few AF_i/g2nc, so 1e-13 of it is covered)
  adjoint lambda: componentwise backward error |J^T lambda - g|_j <=
                  2 sum_i bar_ij |lambda_i| + 1e-13 (|g_j| + sum_i |J_ij lambda_i|)
  dL/dtheta:      first-order propagation of the J bar through the adjoint,
                  sum_ij |lambda_i| bar_ij |mu_j| with mu = J^{-1} dF/dtheta, plus
                  1e-7 relative for the two independent solves' stopping points."""
import numpy as np
import pytest

import adjoint_ref as R
from gpu_util import column_index, entries_ok, n_unknowns, orders, to_dev, to_host

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def dse():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import paper_1206_1779_gb300 as m
    m.load(build_if_missing=True)
    return m


CASES = {
    "tiny": dict(n_cheb=2, n_radial=4, n_angular=4),
    "ragged": dict(n_cheb=13, n_radial=37, n_angular=45),
    "ghost_point": dict(n_cheb=7, n_radial=30, n_angular=33, x_G=3e-3, ginv_G=0.02, x_Z=4e4),
    "constant_extrap": dict(n_cheb=8, n_radial=24, n_angular=32, extrap_mode=1, zinv_Z=2.5),
    "narrow_range": dict(n_cheb=11, n_radial=40, n_angular=64, eps2=1e-3, lambda2=1e3, x_Z=1e3),
    "decoupling_n16": dict(n_cheb=16, n_radial=64, n_angular=32, ginv_G=0.01),
    "n100": dict(n_cheb=100, n_radial=64, n_angular=32),
    "orders_24_48": dict(n_cheb=24, n_cheb_G=48, n_radial=40, n_angular=24, ginv_G=0.01),
    "orders_13_6_ghost_point": dict(n_cheb=13, n_cheb_G=6, n_radial=30, n_angular=33, x_G=3e-3, ginv_G=0.02),
    "paper_quadrature": dict(n_cheb=9, n_cheb_G=7, n_radial=14, n_angular=24, radial_mode=1, angular_mode=1,
                             ginv_G=0.01),
}


def matrix_bar(oracle, p, c):
    Jo, Fo = oracle.newton_matrix(p, c)
    A, AF = oracle.newton_matrix_magnitudes(p, c)
    j = column_index(p).astype(np.float64)
    bar = 1e-11 * np.abs(Jo) + (1e-13 + 16.0 * j[None, :] ** 2 * U) * A
    return Jo, Fo, AF, bar


@pytest.mark.parametrize("name", list(CASES))
def test_vjp_parity(dse, oracle, inputs, name):
    p = inputs.problem(**CASES[name])
    c = inputs.starting_guess(p, seed=21)
    n = n_unknowns(p)
    v = np.random.default_rng(3).standard_normal(n)
    with dse.Plan(p) as plan:
        F = to_dev(np.zeros(n))
        out = to_host(plan.vjp(to_dev(c), to_dev(v), F=F))
        F = to_host(F)
        assert plan.status() == dse.DSE_OK
    Jo, Fo, AF, bar = matrix_bar(oracle, p, c)
    ref = Jo.T @ v
    bound = np.abs(v) @ bar + 4.0 * n * U * (np.abs(v) @ np.abs(Jo))
    err = np.abs(out - ref)
    assert np.all(err <= bound), (name, float(np.max(err / bound)))
    assert all(entries_ok(F, Fo, AF)[:2])


@pytest.mark.parametrize("name", list(CASES))
def test_param_derivatives_parity(dse, oracle, inputs, name):
    p = inputs.problem(**CASES[name])
    c = inputs.starting_guess(p, seed=22)
    n = n_unknowns(p)
    v = np.random.default_rng(4).standard_normal(n)
    with dse.Plan(p) as plan:
        dF = to_host(plan.param_derivatives(to_dev(c)))
        vdF = to_host(plan.param_vjp(to_dev(c), to_dev(v)))
        assert plan.status() == dse.DSE_OK
    dFo = oracle.param_derivatives(p, c)
    _, AF = oracle.newton_matrix_magnitudes(p, c)
    err = np.abs(dF[:, 0] - dFo[:, 0])
    assert np.all(err <= 1e-11 * np.abs(dFo[:, 0]) + 1e-12 * AF / p["g2nc"]), (name, float(np.max(err)))
    assert np.array_equal(dF[:, 1:], dFo[:, 1:])
    ref = v @ dFo
    bound = np.abs(v) @ (1e-11 * np.abs(dFo) + 1e-12 * AF[:, None] / p["g2nc"]) + 4 * n * U * (np.abs(v) @ np.abs(dFo))
    assert np.all(np.abs(vdF - ref) <= bound), (name, vdF, ref)


def test_param_derivatives_reject_zero_coupling(dse, inputs):
    p = inputs.problem(4, 8, 8, g2nc=0.0)
    with dse.Plan(p) as plan:
        with pytest.raises(dse.DseError) as e:
            plan.param_derivatives(to_dev(inputs.starting_guess(inputs.problem(4, 8, 8), seed=1)))
        assert e.value.code == dse.DSE_ERR_ARG


@pytest.mark.parametrize("name", ["tiny", "ragged", "decoupling_n16", "n100", "orders_24_48"])
def test_adjoint_solve_backward_error(dse, oracle, inputs, name):
    p = inputs.problem(**CASES[name])
    c = inputs.starting_guess(p, seed=23)
    n = n_unknowns(p)
    g = np.random.default_rng(5).standard_normal(n)
    with dse.Plan(p) as plan:
        lam_t, st = plan.adjoint_solve(to_dev(c), to_dev(g))
        lam = to_host(lam_t)
    Jo, _, _, bar = matrix_bar(oracle, p, c)
    r = np.abs(Jo.T @ lam - g)
    bound = 2.0 * (np.abs(lam) @ bar) + 1e-13 * (np.abs(g) + np.abs(lam) @ np.abs(Jo))
    assert np.all(r <= bound), (name, float(np.max(r / bound)), st)
    assert st[2] == pytest.approx(np.abs(lam).max(), rel=1e-15)


def test_dressing_vjp_parity(dse, oracle, inputs):
    for extrap, ng in ((0, 0), (1, 0), (0, 17)):
        p = inputs.problem(24, 8, 8, extrap_mode=extrap, n_cheb_G=ng)
        nz, ng = orders(p)
        rng = np.random.default_rng(6)
        # points below eps2, inside, and above lambda2
        x = np.exp(rng.uniform(np.log(1e-9), np.log(1e9), 777))
        gG, gZ = rng.standard_normal(x.size), rng.standard_normal(x.size)
        import torch
        wg = torch.zeros(1, dtype=torch.float64, device="cuda")
        with dse.Plan(p) as plan:
            out = to_host(plan.dressing_vjp(to_dev(x), to_dev(gG), to_dev(gZ), out_g2nc=wg))
            wg = to_host(wg)[0]
            assert plan.status() == dse.DSE_OK
        phi = np.array([oracle.basis(p, xm) for xm in x])
        ref = np.concatenate([phi[:, :nz].T @ gZ, phi[:, :ng].T @ gG])
        mag = np.concatenate([np.abs(phi[:, :nz]).T @ np.abs(gZ), np.abs(phi[:, :ng]).T @ np.abs(gG)])
        j = column_index(p).astype(np.float64)
        assert np.all(np.abs(out - ref) <= (4 * x.size * U + 16 * j ** 2 * U) * mag)
        # d/d g2nc from central differences of the oracle dressing (the UV form is
        # smooth in omega; step 1e-5 relative)
        c = inputs.starting_guess(p, seed=7)
        h = 1e-5 * p["g2nc"]
        pp, pm = dict(p), dict(p)
        pp["g2nc"] += h
        pm["g2nc"] -= h
        gp, zp = oracle.dressing(pp, c, x)
        gm, zm = oracle.dressing(pm, c, x)
        fd = float(gG @ ((gp - gm) / (2 * h)) + gZ @ ((zp - zm) / (2 * h)))
        if extrap == 0:
            assert abs(wg - fd) <= 1e-7 * (np.abs(gG).sum() + np.abs(gZ).sum()) / p["g2nc"]
            assert abs(wg) > 0
        else:
            assert wg == 0.0 and fd == 0.0


def test_dressing_vjp_empty(dse, inputs):
    import torch
    p = inputs.problem(5, 8, 8)
    with dse.Plan(p) as plan:
        e = torch.empty(0, dtype=torch.float64, device="cuda")
        out = to_host(plan.dressing_vjp(e, e, e))
    assert np.array_equal(out, np.zeros(10))


def test_set_couplings_matches_fresh_plan(dse, inputs):
    a = inputs.problem(9, 30, 20)
    b = inputs.problem(9, 30, 20, g2nc=30.0, ginv_G=0.03, zinv_Z=3.0)
    c = to_dev(inputs.starting_guess(a, seed=8))
    with dse.Plan(a) as pa, dse.Plan(b) as pb:
        pa.set_couplings(b["g2nc"], b["ginv_G"], b["zinv_Z"])
        Ja, Fa = pa.newton_matrix(c)
        Jb, Fb = pb.newton_matrix(c)
        assert np.array_equal(to_host(Ja), to_host(Jb))
        assert np.array_equal(to_host(Fa), to_host(Fb))
        with pytest.raises(dse.DseError):
            pa.set_couplings(float("nan"), 0.0, 1.0)


def test_autograd_residual_matches_oracle(dse, oracle, inputs):
    import torch
    from paper_1206_1779_gb300 import autograd as ad
    p = inputs.problem(**CASES["ragged"])
    c = inputs.starting_guess(p, seed=24)
    n = n_unknowns(p)
    v = np.random.default_rng(9).standard_normal(n)
    with dse.Plan(p) as plan:
        ct = to_dev(c).requires_grad_(True)
        theta = torch.tensor([p["g2nc"], p["ginv_G"]], dtype=torch.float64, requires_grad=True)
        F = ad.residual(plan, ct, theta)
        (F * to_dev(v)).sum().backward()
        gc, gt = to_host(ct.grad), theta.grad.numpy()
    Jo, _, AF, bar = matrix_bar(oracle, p, c)
    bound = np.abs(v) @ bar + 4.0 * n * U * (np.abs(v) @ np.abs(Jo))
    assert np.all(np.abs(gc - Jo.T @ v) <= bound)
    dFo = oracle.param_derivatives(p, c)
    ref = v @ dFo[:, :2]
    assert abs(gt[0] - ref[0]) <= 1e-10 * np.abs(v) @ (np.abs(dFo[:, 0]) + AF / p["g2nc"])
    assert gt[1] == pytest.approx(ref[1], rel=1e-14)


def converge_oracle(oracle, p, c, n_relax, rho, tol, max_iter=80):
    for it in range(max_iter):
        c_new, st = oracle.newton_step(p, c, rho if it < n_relax else 1.0)
        if st[1] < tol:
            return c, it
        c = c_new
    raise AssertionError("oracle solve did not converge")


def test_implicit_gradient_full_size(dse, oracle, inputs):
    """N = 64 per function, 256 x 128 nodes, G(x_G)^{-1} = 0.01: the loss over 64
    log-uniform momenta in [1e-4, 1e4] with targets within 5 % of the converged Z,
    differentiated through the solve with respect to (g^2 Nc, G(x_G)^{-1})."""
    import torch
    from paper_1206_1779_gb300 import autograd as ad
    p = inputs.workload_problem("full_solve_n64", ginv_G=0.01)
    N = p["n_cheb"]
    c0 = inputs.starting_guess(p, seed=0)
    x = inputs.loss_momenta(64)
    fac = inputs.target_factors(64)
    tol, rho, n_relax = 1e-11, 0.5, 6
    with dse.Plan(p) as plan:
        theta = torch.tensor([p["g2nc"], p["ginv_G"]], dtype=torch.float64, requires_grad=True)
        xt = to_dev(x)
        cs = ad.solve(plan, theta, to_dev(c0), tol=tol, max_iter=80, rho_relax=rho, n_relax=n_relax)
        _, lZ = ad.dressing(plan, cs, theta, xt)
        Z = torch.exp(lZ)
        t = (Z.detach() * to_dev(fac))
        L = ((Z - t) ** 2).sum()
        L.backward()
        grad = theta.grad.numpy().copy()
        c_star = to_host(cs.detach())

        def loss_at(g2nc, ginv):
            plan.set_couplings(g2nc, ginv, p["zinv_Z"])
            cc = to_dev(c_star)
            plan.solve(cc, tol=tol, max_iter=30)
            lG, lZz = plan.dressing(cc, xt)
            return float(((torch.exp(lZz) - t) ** 2).sum())

        # step 1e-6 max(|theta_k|, 1): the solves stop at the FP64 floor of the
        # residual (~1e-12 dimensionless), so a step of 1e-8 on G(x_G)^{-1} = 0.01
        # would leave the quotient noise-limited at ~1e-4
        fd = []
        for k, name in enumerate(("g2nc", "ginv_G")):
            h = 1e-6 * max(abs(p[name]), 1.0)
            base = [p["g2nc"], p["ginv_G"]]
            up, dn = list(base), list(base)
            up[k] += h
            dn[k] -= h
            fd.append((loss_at(*up) - loss_at(*dn)) / (2 * h))
    fd = np.array(fd)
    # oracle: its own solve, targets and gradient
    co, _ = converge_oracle(oracle, p, c0, n_relax, rho, tol)
    to = R.z_at(oracle, p, co, x) * fac
    go, lam, g = R.implicit_grad(oracle, p, co, x, to)
    Jo, _, _, bar = matrix_bar(oracle, p, co)
    dFo = oracle.param_derivatives(p, co)
    prop = np.array([np.abs(lam) @ bar @ np.abs(oracle.lu_solve(Jo, dFo[:, k])) for k in (0, 1)])
    bound = prop + 1e-7 * np.abs(go[:2])
    print("grad gpu %r fd %r oracle %r bound %r" % (grad.tolist(), fd.tolist(), go[:2].tolist(), bound.tolist()))
    assert np.all(np.abs(grad - fd) <= 1e-5 * np.abs(fd)), (grad, fd)
    assert np.all(np.abs(grad - go[:2]) <= bound), (grad, go[:2], bound)
