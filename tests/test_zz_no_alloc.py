"""dse_residual_static: the allocation-free residual for callers that cannot
call cudaMalloc (device memory owned by another allocator, or no tolerance for
the synchronisation cudaMalloc implies).  It must give the residual of the
plan-based dse_residual, call after call, from its static scratch array.

This file is collected last so that a run that stops at the first failure has
run every other test before it."""
import ctypes

import numpy as np
import pytest

from gpu_util import entries_ok, n_unknowns, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dse():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import paper_1206_1779_gb300 as m
    m.load(build_if_missing=True)
    return m


def static_residual(dse, params, c_dev, F_dev):
    import torch
    L = dse.load()
    prob = dse.Problem.from_params(params)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.dse_residual_static(ctypes.byref(prob), ctypes.c_void_p(c_dev.data_ptr()),
                                 ctypes.c_void_p(F_dev.data_ptr()), stream)


CASES = {
    "newton_step_n16": None,
    "full_solve_n64": None,
    # separate orders (gluon rows at the N_Z roots, ghost rows at the N_G roots) with
    # a ghost subtraction point x_G > 0 (its own row)
    "orders_24_16_ghost_point": dict(n_cheb=24, n_cheb_G=16, n_radial=96, n_angular=64, x_G=2e-3, ginv_G=0.02),
}


@pytest.mark.parametrize("name", list(CASES))
def test_static_residual_matches_plan_residual(dse, oracle, inputs, name):
    import torch
    p = inputs.workload_problem(name) if CASES[name] is None else inputs.problem(**CASES[name])
    _, AF = oracle.newton_matrix_magnitudes(p, inputs.starting_guess(p, seed=0))
    with dse.Plan(p) as plan:
        for seed in (0, 1):  # two calls in a row, different inputs
            c = inputs.starting_guess(p, seed=seed)
            ct = to_dev(c)
            Fp = to_host(plan.residual(ct))
            Fs = torch.full((n_unknowns(p),), float("nan"), dtype=torch.float64, device="cuda")
            assert static_residual(dse, p, ct, Fs) == dse.DSE_OK
            Fs = to_host(Fs)
            r = entries_ok(Fs, Fp, AF)
            assert r.ok, (name, seed, r)


@pytest.mark.parametrize("orders", [(256, 0), (128, 96)])
def test_static_residual_rejects_oversized_problem(dse, inputs, orders):
    import torch
    # 256 coefficients with 4096 x 2048 nodes, and N_Z = 128, N_G = 96 (separate
    # collocation rows) with 512 x 256 nodes, need more than the static scratch
    nz, ng = orders
    p = inputs.problem(nz, 4096, 2048) if ng == 0 else inputs.problem(nz, 512, 256, n_cheb_G=ng)
    n = nz + (ng or nz)
    c = torch.zeros(n, dtype=torch.float64, device="cuda")
    F = torch.zeros(n, dtype=torch.float64, device="cuda")
    assert static_residual(dse, p, c, F) == dse.DSE_ERR_ARG
