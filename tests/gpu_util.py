"""Shared helpers of the GPU parity tests (tolerances, device transfer).

Parity bar for the Newton matrix J and the residual F (per entry):
    |gpu - oracle| <= 1e-11 |oracle| + (1e-13 + 16 j^2 u) A
with u = 2^-53, j the Chebyshev index of the entry's column (0 for F) and A
the sum of the magnitudes of every summand that forms the entry
(oracle.newton_matrix_magnitudes): the -Z^{-1} phi_j term and each quadrature
summand of the row and of its subtraction row.
 - 1e-13 A: entries that are small differences of large terms (the MOM
   subtraction, the cancellation of the quadratic parts of the Q and M terms,
   oscillating phi_j(z)) carry ~1e-16 A of rounding on any FP64 evaluation
   order; 1e-13 A bounds sums of up to ~1e5 terms.
 - 16 j^2 u A: T_j(s) has slope up to j^2 near s = +-1, so the one-ulp
   difference between two implementations of s(z) = (ln z - L0)/L1 (library
   log) and of the recurrence moves phi_j by up to a few j^2 u.
Strict bar, on the entries that are not small differences of large summands
(|oracle| >= 1e-2 A, so that 1e-11 |oracle| >= 1e-13 A):
    |gpu - oracle| <= 1e-11 |oracle| + 16 j^2 u A
i.e. the 1e-11 relative bar with only the allowance for the rounding of s(z) kept.
The fraction of all entries within 1e-11 relative (no floor at all) is reported;
the production-size tests assert a lower bound on it.
"""
from typing import NamedTuple

import numpy as np

REL = 1e-11
ABS_OF_MAGNITUDE = 1e-13
U = 2.0 ** -53


def orders(p):
    """(N_Z, N_G) of a problem dict (n_cheb_G = 0 means N_G = N_Z)."""
    nz = int(p["n_cheb"])
    return nz, int(p.get("n_cheb_G", 0) or 0) or nz


def n_unknowns(p) -> int:
    nz, ng = orders(p)
    return nz + ng


def column_index(p) -> np.ndarray:
    """Chebyshev index of every column of J (a_0..a_{N_Z-1}, b_0..b_{N_G-1})."""
    nz, ng = orders(p)
    return np.concatenate([np.arange(nz), np.arange(ng)])


STRICT_CONDITIONING = 1e-2


class Parity(NamedTuple):
    ok: bool              # every entry within the bar
    strict_ok: bool       # every entry of the strict subset within the strict bar
    nbad: int             # entries outside the bar
    worst: float          # max |gpu - oracle| / A
    strict_ratio: float   # max over the strict subset of err / (1e-11 |O| + 16 j^2 u A)
    n_strict: int         # size of the strict subset
    frac_rel: float       # fraction of all entries with err <= 1e-11 |O|


def entries_ok(G, O, A, jidx=None) -> Parity:
    G, O, A = (np.asarray(a, dtype=np.float64) for a in (G, O, A))
    err = np.abs(G - O)
    j2 = 0.0 if jidx is None else np.asarray(jidx, dtype=np.float64) ** 2
    j2 = np.broadcast_to(j2, O.shape)
    ok = err <= REL * np.abs(O) + (ABS_OF_MAGNITUDE + 16.0 * j2 * U) * A
    # (an entry with A = 0 has no summand: it must be exactly 0 on both sides)
    strict = (np.abs(O) >= STRICT_CONDITIONING * A) & (A > 0)
    sbar = REL * np.abs(O) + 16.0 * j2 * U * A
    sratio = float(np.max(err[strict] / sbar[strict])) if strict.any() else 0.0
    frac = float(np.mean(err <= REL * np.abs(O))) if O.size else 1.0
    pos = A > 0
    worst = float(np.max(err[pos] / A[pos])) if pos.any() else 0.0
    return Parity(bool(ok.all()), sratio <= 1.0, int((~ok).sum()), worst, sratio, int(strict.sum()), frac)


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
