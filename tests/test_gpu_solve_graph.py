"""The Newton iteration of dse_solve as one CUDA graph (a while node whose body is
one Newton step and a decision kernel) against the host-driven loop that an
instrumented plan (dse_plan_profile on) keeps: the same kernels in the same
order, so coefficients, step counts and stats agree bit for bit, for the
relaxed and mixed-precision iterations (whose first steps stay on the host),
at the step limit, on a non-finite status and after a change of couplings."""
import numpy as np
import pytest

from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dse():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import paper_1206_1779_gb300 as m
    m.load(build_if_missing=True)
    return m


def _solve(dse, plan, c, host_loop, **kw):
    """(coefficients, iterations, stats, error code or 0, kernels launched)."""
    plan.profile(host_loop)
    ct = to_dev(c)
    l0 = plan.counters()[0]
    code, it, st = 0, None, None
    try:
        it, st = plan.solve(ct, **kw)
    except dse.DseError as e:
        code = e.code
    l1 = plan.counters()[0]
    plan.profile(False)
    return to_host(ct), it, st, code, l1 - l0


@pytest.mark.parametrize("name", ["newton_step_n16", "full_solve_n64"])
def test_graph_solve_matches_host_loop(dse, inputs, name):
    p = inputs.workload_problem(name)
    c = inputs.starting_guess(p, seed=0)
    with dse.Plan(p) as plan:
        ch, ith, sth, codeh, lh = _solve(dse, plan, c, True, tol=1e-10, max_iter=50)
        cg, itg, stg, codeg, lg = _solve(dse, plan, c, False, tol=1e-10, max_iter=50)
        # a second graph solve replays the instantiated graph
        cg2, itg2, _, _, lg2 = _solve(dse, plan, c, False, tol=1e-10, max_iter=50)
    assert codeh == 0 and codeg == 0
    assert sth[1] < 1e-10
    assert ith == itg == itg2
    assert np.array_equal(ch, cg) and np.array_equal(cg, cg2)
    assert sth == stg
    # the graph adds the copy-in and copy-out kernels and one decision kernel per step
    assert lg == lh + 2 + itg and lg2 == lg, (lh, lg, lg2, itg)


def test_graph_solve_relaxed_steps(dse, inputs):
    # the relaxed steps (rho = 0.5) run on the host, the rest in the graph
    p = inputs.workload_problem("newton_step_n16")
    c = inputs.starting_guess(p, seed=1)
    kw = dict(tol=1e-10, max_iter=60, rho_relax=0.5, n_relax=4)
    with dse.Plan(p) as plan:
        ch, ith, sth, codeh, _ = _solve(dse, plan, c, True, **kw)
        cg, itg, stg, codeg, _ = _solve(dse, plan, c, False, **kw)
    assert codeh == codeg == 0
    assert ith == itg and ith > 4
    assert np.array_equal(ch, cg) and sth == stg


def test_graph_solve_mixed_precision(dse, inputs):
    # FP32 residuals on the host until the switch to FP64 residuals, then the graph
    p = inputs.workload_problem("full_solve_n64", precision=1)
    c = inputs.starting_guess(p, seed=0)
    with dse.Plan(p) as plan:
        ch, ith, sth, codeh, _ = _solve(dse, plan, c, True, tol=1e-10, max_iter=50)
        cg, itg, stg, codeg, _ = _solve(dse, plan, c, False, tol=1e-10, max_iter=50)
    assert codeh == codeg == 0
    assert ith == itg and np.array_equal(ch, cg) and sth == stg


def test_graph_solve_step_limit(dse, inputs):
    p = inputs.problem(6, 16, 16)
    c = inputs.starting_guess(p, seed=0)
    with dse.Plan(p) as plan:
        ch, _, _, codeh, _ = _solve(dse, plan, c, True, tol=1e-10, max_iter=2)
        cg, _, _, codeg, _ = _solve(dse, plan, c, False, tol=1e-10, max_iter=2)
        # the limit may also fall inside the graph after host-driven relaxed steps
        cr, _, _, coder, _ = _solve(dse, plan, c, False, tol=1e-10, max_iter=3, rho_relax=0.5, n_relax=2)
        crh, _, _, coderh, _ = _solve(dse, plan, c, True, tol=1e-10, max_iter=3, rho_relax=0.5, n_relax=2)
    assert codeh == codeg == coder == coderh == dse.DSE_ERR_NOT_CONVERGED
    assert np.array_equal(ch, cg) and np.array_equal(cr, crh)
    assert not np.array_equal(ch, c)


def test_graph_solve_nonfinite_status(dse, inputs):
    p = inputs.workload_problem("newton_step_n16")
    c = inputs.starting_guess(p, seed=0)
    bad = c.copy()
    bad[3] = float("nan")
    with dse.Plan(p) as plan:
        cb, _, _, code, _ = _solve(dse, plan, bad, False, tol=1e-10, max_iter=50)
        assert code == dse.DSE_ERR_NONFINITE
        assert plan.status() == 0  # the status word was cleared
        # coefficients untouched; the plan (and its graph) stays usable
        assert np.isnan(cb[3]) and np.array_equal(np.delete(cb, 3), np.delete(bad, 3))
        cg, itg, stg, codeg, _ = _solve(dse, plan, c, False, tol=1e-10, max_iter=50)
        ch, ith, sth, codeh, _ = _solve(dse, plan, c, True, tol=1e-10, max_iter=50)
    assert codeg == codeh == 0 and itg == ith and np.array_equal(cg, ch) and stg == sth


def test_graph_solve_after_new_couplings(dse, inputs):
    # the graph's kernels hold the couplings: a change rebuilds it
    p = inputs.workload_problem("newton_step_n16")
    c = inputs.starting_guess(p, seed=0)
    with dse.Plan(p) as plan:
        c0, _, _, code0, _ = _solve(dse, plan, c, False, tol=1e-10, max_iter=50)
        plan.set_couplings(p["g2nc"] * 1.01, p["ginv_G"], p["zinv_Z"])
        cg, itg, stg, codeg, _ = _solve(dse, plan, c, False, tol=1e-10, max_iter=50)
        ch, ith, sth, codeh, _ = _solve(dse, plan, c, True, tol=1e-10, max_iter=50)
    assert code0 == codeg == codeh == 0
    assert itg == ith and np.array_equal(cg, ch) and stg == sth
    assert not np.array_equal(cg, c0)
