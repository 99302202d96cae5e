"""Host-side pins for the constants of the Schwinger-function cosine
(dse_kernels.cu): the two-part pi/2 of the Cody-Waite reduction, 2/pi and the
rounding shifter, checked against 50-digit arithmetic; and the tail-coefficient
recurrence of the kernel (the factorials (2k+4)!, (2k+5)! it builds by products)."""
import math
import os
import re

import pytest

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_1206_1779_gb300", "csrc", "dse_kernels.cu")


def constant(name):
    m = re.search(r"constexpr double %s = ([-0-9.eE+]+);" % name, open(SRC).read())
    assert m, name
    return float(m.group(1))


def test_reduction_constants():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    half_pi = mpmath.pi / 2
    p1, p2 = constant("kPio2_1"), constant("kPio2_2")
    assert p1 == float(half_pi)
    assert p2 == float(half_pi - mpmath.mpf(p1))
    # the two parts carry pi/2 to 1.5e-33: k below 2^50 leaves an error under 2e-18
    rem = abs(mpmath.mpf(p1) + mpmath.mpf(p2) - half_pi)
    assert rem < 1.5e-33 and rem * 2 ** 50 < 2e-18
    assert constant("kTwoOverPi") == float(2 / mpmath.pi)
    assert constant("kRoundShifter") == 1.5 * 2.0 ** 52


def test_tail_factorials():
    # the kernel starts from 4! and 5! and multiplies by (2k+5)(2k+6), (2k+6)(2k+7)
    fc, fs = 24.0, 120.0
    for k in range(8):
        assert fc == math.factorial(2 * k + 4) and fs == math.factorial(2 * k + 5)
        fc *= (2 * k + 5) * (2 * k + 6)
        fs *= (2 * k + 6) * (2 * k + 7)
    # truncation after the r^18 (cos) and r^19 (sin) terms at |r| = pi/4
    r = math.pi / 4
    assert r ** 20 / math.factorial(20) < 4e-21 and r ** 21 / math.factorial(21) < 4e-21
