"""Mixed-precision mode (precision = 1): the Newton matrix from FP32 integrands
with FP64 block accumulation, the residual in FP64, and the Newton iteration
that pairs them (an inexact Newton method whose fixed point is the FP64
solution).  Reported against the FP64 oracle: the Newton-matrix error per entry
and the converged dressing functions (target 1e-8)."""
import math

import numpy as np
import pytest

from gpu_util import entries_ok, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dse():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import paper_1206_1779_gb300 as m
    m.load(build_if_missing=True)
    return m


@pytest.mark.parametrize("name", ["newton_step_n16", "full_solve_n64", "matrix_n128"])
def test_mixed_newton_matrix_error(dse, oracle, inputs, name):
    p64 = inputs.workload_problem(name)
    p32 = dict(p64, precision=1)
    c = inputs.starting_guess(p64, seed=0)
    with dse.Plan(p32) as plan:
        J, F = plan.newton_matrix(to_dev(c))
        J, F = to_host(J), to_host(F)
        Fr = to_host(plan.residual(to_dev(c)))
    Jo, Fo = oracle.newton_matrix(p64, c)
    A, AF = oracle.newton_matrix_magnitudes(p64, c)
    # the residual is FP64 in both calls: the full parity bar
    assert all(entries_ok(F, Fo, AF)[:2])
    assert all(entries_ok(Fr, Fo, AF)[:2])
    # the FP32-integrand Jacobian: error per entry relative to its magnitude sum
    rel = np.abs(J - Jo) / A
    big = np.abs(Jo) >= 1e-2 * A  # entries that are not small differences of large summands
    relJ = np.abs(J - Jo)[big] / np.abs(Jo[big])
    print("%s: max |dJ|/A = %.2e, median %.2e; |dJ|/|J| over the %d of %d entries with |J| >= 1e-2 A: "
          "max %.2e, median %.2e" % (name, rel.max(), np.median(rel), big.sum(), J.size, relJ.max(),
                                      np.median(relJ)))
    assert rel.max() < 1e-5
    assert relJ.max() < 1e-3


@pytest.mark.parametrize("name", ["newton_step_n16", "full_solve_n64", "matrix_n128"])
def test_mixed_solve_reaches_fp64_solution(dse, oracle, inputs, name):
    p64 = inputs.workload_problem(name)
    p32 = dict(p64, precision=1)
    c0 = inputs.starting_guess(p64, seed=0)
    co, ito, _ = oracle.solve(p64, c0, tol=1e-10)
    x = np.exp(np.linspace(math.log(1e-6), math.log(1e6), 97))
    with dse.Plan(p32) as plan:
        ct = to_dev(c0)
        it, st = plan.solve(ct, tol=1e-10, max_iter=40)
        gG, gZ = plan.dressing(ct, to_dev(x))
        gG, gZ = to_host(gG), to_host(gZ)
    assert st[1] < 1e-10
    lG, lZ = oracle.dressing(p64, co, x)
    dG, dZ = np.max(np.abs(gG - lG)), np.max(np.abs(gZ - lZ))
    print("%s: %d mixed iterations (oracle %d); max |d ln G| %.2e, |d ln Z| %.2e" % (name, it, ito + 1, dG, dZ))
    assert dG < 1e-8 and dZ < 1e-8
    assert it <= ito + 6
