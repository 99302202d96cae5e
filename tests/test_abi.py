"""Host-side checks of the C ABI (no GPU work): the library loads, exports every
entry point declared in include/*.h, and rejects bad arguments before
touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1206_1779_gb300 import build, load
    build.build()
    return load()


def declared_functions():
    inc = os.path.join(ROOT, "include")
    src = "\n".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dse_[a-z_]+)\s*\(", src)))


def test_exports_match_header(lib):
    from paper_1206_1779_gb300 import EXPORTS
    names = declared_functions()
    assert set(names) == set(EXPORTS)
    for n in names:
        assert hasattr(lib, n), n


def test_struct_layout_matches_header(tmp_path):
    """Size and field offsets of dse_problem as a C compiler lays it out from
    include/dse.h, against the ctypes mirror of the binding."""
    import os
    import subprocess
    from paper_1206_1779_gb300 import Problem
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    names = [n for n, _ in Problem._fields_]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "dse.h"', 'int main(void) {',
             '    printf("size %zu\\n", sizeof(dse_problem));']
    lines += ['    printf("' + n + ' %zu\\n", offsetof(dse_problem, ' + n + '));' for n in names]
    lines += ['    return 0;', '}', '']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(root, "include"), "-o", str(exe), str(src)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                       text=True).stdout.splitlines())
    assert int(out["size"]) == ctypes.sizeof(Problem)
    for n in names:
        assert int(out[n]) == getattr(Problem, n).offset, n


def test_status_strings(lib):
    for code in [0, -1, -2, -3, -4, -5, -6]:
        assert lib.dse_status_string(code)
    assert lib.dse_status_string(-99) == b"unknown status"


@pytest.mark.parametrize("bad", [dict(n_cheb=0), dict(n_cheb=300), dict(n_radial=0), dict(n_angular=-3),
                                 dict(eps2=0.0), dict(lambda2=1e-9), dict(x_Z=0.0), dict(x_G=-1.0),
                                 dict(g2nc=float("nan"))])
def test_plan_create_rejects_bad_problem(lib, inputs, bad):
    from paper_1206_1779_gb300 import DSE_ERR_ARG, Problem
    p = inputs.problem(8, 16, 16)
    p.update(bad)
    prob = Problem.from_params(p)
    h = ctypes.c_void_p(123)
    assert lib.dse_plan_create(ctypes.byref(prob), None, ctypes.byref(h)) == DSE_ERR_ARG
    assert not h.value


def test_plan_create_rejects_unsupported_modes(lib, inputs):
    from paper_1206_1779_gb300 import DSE_ERR_UNSUPPORTED, Problem
    for over in [dict(radial_mode=2), dict(precision=2), dict(extrap_mode=7), dict(angular_mode=3)]:
        p = inputs.problem(8, 16, 16)
        p.update(over)
        h = ctypes.c_void_p()
        assert lib.dse_plan_create(ctypes.byref(Problem.from_params(p)), None, ctypes.byref(h)) == DSE_ERR_UNSUPPORTED


def test_null_plan_arguments(lib):
    from paper_1206_1779_gb300 import DSE_ERR_ARG, DSE_OK
    assert lib.dse_plan_create(None, None, None) == DSE_ERR_ARG
    assert lib.dse_plan_destroy(None) == DSE_OK
    assert lib.dse_residual(None, None, None) == DSE_ERR_ARG
    assert lib.dse_newton_matrix(None, None, None, None) == DSE_ERR_ARG
    assert lib.dse_newton_step(None, None, 1.0, None) == DSE_ERR_ARG
    assert lib.dse_schwinger(None, None, None, 0, 1, None) == DSE_ERR_ARG
    assert lib.dse_plan_status(None) == DSE_ERR_ARG


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1206_1779_gb300 import _binding
    monkeypatch.setattr(_binding, "_lib", None)
    monkeypatch.setattr(_binding._build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        _binding.load()


def test_alu_peak_rejects_bad_arguments(lib):
    import ctypes as C
    rate = C.c_double()
    # checked before any device work
    assert lib.dse_alu_peak(9, 100.0, None, C.byref(rate), None) == -1
    assert lib.dse_alu_peak(0, 0.5, None, C.byref(rate), None) == -1
    assert lib.dse_alu_peak(0, float("nan"), None, C.byref(rate), None) == -1
    assert lib.dse_alu_peak(0, 100.0, None, None, None) == -1


def test_static_residual_rejects_unsupported_modes(lib):
    """The allocation-free residual refuses the split radial rule and mixed
    precision, and oversized problems, before any device work."""
    import ctypes as C
    from paper_1206_1779_gb300 import Problem, inputs
    for over, code in ((dict(radial_mode=1), -5), (dict(precision=1), -5)):
        prob = Problem.from_params(inputs.problem(8, 16, 16, **over))
        assert lib.dse_residual_static(C.byref(prob), C.c_void_p(16), C.c_void_p(16), None) == code
    prob = Problem.from_params(inputs.problem(128, 512, 256, n_cheb_G=96))
    assert lib.dse_residual_static(C.byref(prob), C.c_void_p(16), C.c_void_p(16), None) == -1
