"""Fit error of the piecewise-polynomial table of the dressing functions that the
FP64 quadrature kernel reads in place of the per-triple Chebyshev sums (Sec. 3:
ln G, ln Z are Chebyshev series in s(x)), for every order the kernel uses it at,
24 <= N <= 256.

The table splits s in [-1, 1] into M = 256 intervals uniform in theta = arccos s;
on each it interpolates a function at the Q = 16 Chebyshev points of
u = (s - mid)/half, i.e. a polynomial of degree 15 in s.  The interpolation is
linear in the function, so for ln Z = a_0/2 + sum_j a_j T_j(s) its error is the
sum of the errors of the modes T_j weighted by |a_j|; modes j <= 15 are
polynomials of degree <= 15 and are reproduced exactly.  The bound pinned here,
for the interval width h = pi/M,

    max over intervals and u of |I[T_j] - T_j| <= 4 (j h/4)^16 / 16!,

gives for the table of Z = e^(ln Z) (and likewise G, W = G^p Z^q) a relative
error below 4 (N h/4)^16/16! * sum_{j>=16} |a_j| to first order: 3.8e-15 times
that sum at N = 256, 1e-17 at N = 192, 1e-24 at N = 64.  The emulation below
follows the table's definition (intervals, nodes, interpolation), not the
kernel's code; the GPU parity tests at N = 192 and 256 check the kernel.
"""
import math

import numpy as np
import pytest

M = 256
Q = 16


def _interval(i, mp=None):
    if mp is None:
        th0, th1 = i * math.pi / M, (i + 1) * math.pi / M
        return 0.5 * (math.cos(th0) + math.cos(th1)), 0.5 * (math.cos(th0) - math.cos(th1))
    th0, th1 = i * mp.pi / M, (i + 1) * mp.pi / M
    return (mp.cos(th0) + mp.cos(th1)) / 2, (mp.cos(th0) - mp.cos(th1)) / 2


def _bound(j: int) -> float:
    return 4.0 * (j * math.pi / M / 4.0) ** 16 / math.factorial(16)


@pytest.mark.parametrize("j", [3, 15, 16, 24, 64, 128, 192, 255])
def test_mode_interpolation_bound(j):
    """Per-mode interpolation error in 45-digit arithmetic, on every fourth interval
    and the two at each end (where arccos is steepest)."""
    mp = pytest.importorskip("mpmath").mp
    mp.dps = 45
    uq = [mp.cos(mp.pi * (q + mp.mpf(1) / 2) / Q) for q in range(Q)]
    dct = [[mp.cos(mp.pi * k * (r + mp.mpf(1) / 2) / Q) for r in range(Q)] for k in range(Q)]
    tu = [mp.mpf(-1) + mp.mpf(k) / 8 for k in range(17)]
    worst = mp.mpf(0)
    for i in sorted(set(list(range(0, M, 4)) + [1, 2, M - 2, M - 1])):
        mid, half = _interval(i, mp)
        v = [mp.cos(j * mp.acos(mid + half * u)) for u in uq]
        ck = [(2 if k else 1) * mp.fsum(v[r] * dct[k][r] for r in range(Q)) / Q for k in range(Q)]
        for u in tu:
            p = mp.fsum(ck[k] * mp.cos(k * mp.acos(u)) for k in range(Q))
            worst = max(worst, abs(p - mp.cos(j * mp.acos(mid + half * u))))
    if j <= 15:
        assert worst < mp.mpf(10) ** -40  # a polynomial of degree <= 15: exact
    else:
        assert worst <= _bound(j), (j, float(worst), _bound(j))
        # and, beyond the first modes, not loose by orders of magnitude
        if j >= 24:
            assert worst >= _bound(j) / 16, (j, float(worst), _bound(j))


def _cheb_series(c, s):
    """c_0/2 + sum_j c_j T_j(s) (Clenshaw)."""
    b1 = np.zeros_like(s)
    b2 = np.zeros_like(s)
    for k in range(len(c) - 1, 0, -1):
        b1, b2 = c[k] + 2 * s * b1 - b2, b1
    return c[0] / 2 + s * b1 - b2


@pytest.mark.parametrize("N", [64, 192, 256])
def test_dressing_table_fit(inputs, N):
    """Z, G and W = G^p Z^q of the seeded coefficient vectors the parity tests use
    (the starting guess plus 0.01 N(0,1)/(j+1) in every mode), fitted on every
    interval as the table defines it and compared with the series between the
    nodes, all in numpy's extended precision (64-bit significand on x86-64), which
    resolves relative errors down to ~1e-18 |ln F|."""
    ld = np.longdouble
    if np.finfo(ld).eps > 1e-18:
        pytest.skip("needs an extended-precision long double")
    p = inputs.problem(N, 256, 128)
    c = inputs.starting_guess(p, seed=0).astype(ld)
    a, b = c[:N], c[N:]
    delta = ld(p["delta"])
    pexp, qexp = -2 - 6 * delta, -3 * delta
    pi = ld(np.pi) + ld(1.2246467991473531772e-16)  # pi to extended precision
    uq = np.cos(pi * (np.arange(Q, dtype=ld) + ld(0.5)) / Q)
    ut = np.linspace(ld(-1), ld(1), 41, dtype=ld)
    Tq = np.cos(np.outer(np.arange(Q, dtype=ld), np.arccos(uq)))  # T_k(u_q)
    Tt = np.cos(np.outer(np.arange(Q, dtype=ld), np.arccos(ut)))
    worst = 0.0
    for i in range(M):
        th0, th1 = i * pi / M, (i + 1) * pi / M
        mid, half = (np.cos(th0) + np.cos(th1)) / 2, (np.cos(th0) - np.cos(th1)) / 2
        sq, st = mid + half * uq, mid + half * ut
        lzq, lgq = _cheb_series(a, sq), _cheb_series(b, sq)
        lzt, lgt = _cheb_series(a, st), _cheb_series(b, st)
        for lq, lt in ((lzq, lzt), (lgq, lgt), (pexp * lgq + qexp * lzq, pexp * lgt + qexp * lzt)):
            ck = (ld(2) / Q) * (Tq @ np.exp(lq))
            ck[0] /= 2
            fit = ck @ Tt
            ft = np.exp(lt)
            rel = float(np.max(np.abs(fit - ft) / ft)) / max(1.0, float(np.max(np.abs(lt))))
            worst = max(worst, rel)
    tail = float(np.sum(np.abs(np.concatenate([a[16:], b[16:]]))))
    print("N=%d: worst relative fit error / max(1, |ln F|) = %.2e; mode bound x tail = %.2e"
          % (N, worst, _bound(N) * tail))
    assert _bound(N) * tail < 1e-15
    assert worst < max(4.0 * _bound(N) * tail, 1e-17)
