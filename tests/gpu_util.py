"""Shared helpers of the GPU parity tests (tolerances, device transfer)."""
import numpy as np

# Per-entry bar: relative 1e-11, with an absolute floor of 1e-13 times the
# row's largest |J| for entries that are small through cancellation (the
# subtraction at x_Z / x_G and the quadratic-divergence cancellation between
# the Q and M terms bound their relative precision).
REL = 1e-11
ROW_FLOOR = 1e-13


def matrix_ok(J, Jo):
    rowmax = np.abs(Jo).max(axis=1, keepdims=True)
    err = np.abs(J - Jo)
    ok = err <= REL * np.abs(Jo) + ROW_FLOOR * rowmax
    big = np.abs(Jo) > 1e-6 * rowmax
    rel = float(np.max(err[big] / np.abs(Jo[big]))) if big.any() else 0.0
    return bool(ok.all()), rel, int((~ok).sum())


def residual_ok(F, Fo, Jo):
    rowmax = np.abs(Jo).max(axis=1)
    err = np.abs(F - Fo)
    ok = err <= REL * np.abs(Fo) + ROW_FLOOR * rowmax
    return bool(ok.all()), float(np.max(err / (np.abs(Fo) + ROW_FLOOR * rowmax)))


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def to_host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()
