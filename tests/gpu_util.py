"""Shared helpers of the GPU parity tests (tolerances, device transfer).

Parity bar for the Newton matrix J and the residual F (per entry):
    |gpu - oracle| <= 1e-11 |oracle| + 1e-13 A
where A is the sum of the magnitudes of every summand that forms the entry
(oracle.newton_matrix_magnitudes): the -Z^{-1} phi_j term and each quadrature
summand of the row and of its subtraction row.  Entries that are small
differences of large terms (the MOM subtraction, the cancellation of the
quadratic parts of the Q and M terms, oscillating phi_j(z)) cannot be
reproduced to 1e-11 relative by any FP64 evaluation that rounds differently,
because each side carries ~1e-16 A of rounding; 1e-13 A bounds sums of up to
~1e5 terms.  Well-conditioned entries (|J| >= 1e-3 A) are held to 1e-11
relative by the first term alone; the tests also report their largest
relative error.
"""
import numpy as np

REL = 1e-11
ABS_OF_MAGNITUDE = 1e-13


def entries_ok(G, O, A):
    err = np.abs(G - O)
    ok = err <= REL * np.abs(O) + ABS_OF_MAGNITUDE * A
    well = np.abs(O) >= 1e-3 * A
    rel_well = float(np.max(err[well] / np.abs(O[well]))) if well.any() else 0.0
    return bool(ok.all()), rel_well, int((~ok).sum()), float(np.max(err / A))


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def to_host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def dump(name, **arrays):
    """Save arrays for offline analysis when DSE_TEST_DUMP names a directory."""
    import os
    d = os.environ.get("DSE_TEST_DUMP")
    if d:
        os.makedirs(d, exist_ok=True)
        np.savez(os.path.join(d, name + ".npz"), **arrays)
