"""The arithmetic-rate microbenchmark that the roofline divides by (dse_alu_peak):
each pipe's measured rate is positive, repeatable, and in the ratio the
datasheet's unit counts give (FP32 FMA 64 times FP64 FMA on this GPU; the
special-function unit well below FP32 FMA), so that a rate that measured the
wrong instruction or a launch that did no work would fail."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dse():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import paper_1206_1779_gb300 as m
    m.load(build_if_missing=True)
    return m


def test_alu_peaks(dse):
    r = {}
    for name, kind in (("fp64", dse.DSE_PEAK_FP64_FMA), ("fp32", dse.DSE_PEAK_FP32_FMA),
                       ("ex2", dse.DSE_PEAK_MUFU_EX2), ("lg2", dse.DSE_PEAK_MUFU_LG2),
                       ("dmma", dse.DSE_PEAK_FP64_DMMA), ("fp32x2", dse.DSE_PEAK_FP32X2_FMA)):
        a, ms_a = dse.alu_peak(kind, 20.0)
        b, ms_b = dse.alu_peak(kind, 20.0)
        assert a > 0 and b > 0 and 5.0 < ms_a < 200.0, (name, a, ms_a)
        assert abs(a / b - 1.0) < 0.2, (name, a, b)
        r[name] = max(a, b)
    print("FMA/s: FP64 %.3e, FP32 %.3e, FP32 paired %.3e, FP64 tensor (DMMA) %.3e; exp2/s %.3e, log2/s %.3e"
          % (r["fp64"], r["fp32"], r["fp32x2"], r["dmma"], r["ex2"], r["lg2"]))
    # the paired instruction does two FMAs: at least the scalar rate, at most twice it
    assert 0.8 * r["fp32"] < r["fp32x2"] < 2.5 * r["fp32"]
    assert 16.0 < r["fp32"] / r["fp64"] < 256.0
    assert r["ex2"] < r["fp32"] and r["lg2"] < r["fp32"]
    # the FP64 tensor path is an FP64 unit too: within a small factor of the FP64 FMA pipe
    assert r["fp64"] / 16.0 < r["dmma"] < 16.0 * r["fp64"]
