"""ctypes front end of the FP64 CPU oracle (oracle/dse_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module; the product package
never does.  The oracle follows arXiv:1206.1779 Sec. 2 (equations, kernels,
asymptotics, MOM subtraction) and Sec. 3 (Chebyshev expansion, collocation,
Newton matrix) in plain double precision; see the header of dse_oracle.h.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dse_oracle.c")
_HDR = os.path.join(_HERE, "dse_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libdse_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE double, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Problem(ctypes.Structure):
    _fields_ = [
        ("n_cheb", ctypes.c_int), ("n_radial", ctypes.c_int), ("n_angular", ctypes.c_int),
        ("eps2", ctypes.c_double), ("lambda2", ctypes.c_double), ("g2nc", ctypes.c_double),
        ("x_G", ctypes.c_double), ("ginv_G", ctypes.c_double),
        ("x_Z", ctypes.c_double), ("zinv_Z", ctypes.c_double),
        ("kappa", ctypes.c_double), ("delta", ctypes.c_double),
        ("radial_mode", ctypes.c_int), ("extrap_mode", ctypes.c_int), ("precision", ctypes.c_int),
        ("n_cheb_G", ctypes.c_int), ("angular_mode", ctypes.c_int),
    ]


_D = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.POINTER(Problem)
            sig = {
                "dse_ref_gauss_legendre": [ctypes.c_int, _D, _D],
                "dse_ref_quadrature": [P, _D, _D, _D, _D],
                "dse_ref_radial_rule": [P, ctypes.c_double, _D, _D],
                "dse_ref_collocation": [P, _D],
                "dse_ref_collocation_ghost": [P, _D],
                "dse_ref_basis": [P, ctypes.c_double, _D],
                "dse_ref_dressing": [P, _D, ctypes.c_int, _D, _D, _D],
                "dse_ref_kernels": [ctypes.c_double, ctypes.c_double, ctypes.c_double, _D, _D, _D],
                "dse_ref_self_energy": [P, _D, ctypes.c_double, _D, _D, _D, _D],
                "dse_ref_residual": [P, _D, _D],
                "dse_ref_newton_matrix": [P, _D, _D, _D],
                "dse_ref_newton_matrix_magnitudes": [P, _D, _D, _D],
                "dse_ref_param_derivatives": [P, _D, _D],
                "dse_ref_lu_solve": [ctypes.c_int, _D, _D, _D],
                "dse_ref_newton_step": [P, _D, ctypes.c_double, _D],
                "dse_ref_schwinger_nodes": [P, ctypes.c_int, _D, _D],
                "dse_ref_schwinger": [P, _D, _D, ctypes.c_int, ctypes.c_int, _D],
                "dse_ref_num_threads": [],
            }
            for name, args in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = ctypes.c_int
            L.dse_ref_map.argtypes = [P, ctypes.c_double]
            L.dse_ref_map.restype = ctypes.c_double
            _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


def _chk(st: int, what: str) -> None:
    if st != 0:
        raise OracleError("%s failed with status %d" % (what, st))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def make_problem(params: dict) -> Problem:
    p = Problem()
    for name, _ in Problem._fields_:
        setattr(p, name, params.get(name, 0))
    return p


def orders(params: dict):
    """(N_Z, N_G): Chebyshev orders of ln Z and ln G (n_cheb_G = 0 means N_G = N_Z)."""
    nz = int(params["n_cheb"])
    ng = int(params.get("n_cheb_G", 0) or 0)
    return nz, (ng if ng > 0 else nz)


def n_unknowns(params: dict) -> int:
    nz, ng = orders(params)
    return nz + ng


def gauss_legendre(n: int):
    x = np.empty(n); w = np.empty(n)
    _chk(lib().dse_ref_gauss_legendre(n, _ptr(x), _ptr(w)), "gauss_legendre")
    return x, w


def radial_count(params: dict) -> int:
    return (3 if params.get("radial_mode", 0) == 1 else 1) * int(params["n_radial"])


def radial_rule(params: dict, x: float):
    """Radial nodes and weights used for external momentum x."""
    p = make_problem(params)
    n = radial_count(params)
    y = np.empty(n); W = np.empty(n)
    _chk(lib().dse_ref_radial_rule(ctypes.byref(p), float(x), _ptr(y), _ptr(W)), "radial_rule")
    return y, W


def quadrature(params: dict):
    p = make_problem(params)
    n = radial_count(params)
    y = np.empty(n); W = np.empty(n)
    th = np.empty(p.n_angular); wt = np.empty(p.n_angular)
    _chk(lib().dse_ref_quadrature(ctypes.byref(p), _ptr(y), _ptr(W), _ptr(th), _ptr(wt)), "quadrature")
    return y, W, th, wt


def collocation(params: dict, ghost: bool = False) -> np.ndarray:
    """Gluon collocation points (N_Z), or the ghost points (N_G) with ghost=True."""
    p = make_problem(params)
    nz, ng = orders(params)
    if ghost:
        x = np.empty(ng)
        _chk(lib().dse_ref_collocation_ghost(ctypes.byref(p), _ptr(x)), "collocation_ghost")
    else:
        x = np.empty(nz)
        _chk(lib().dse_ref_collocation(ctypes.byref(p), _ptr(x)), "collocation")
    return x


def map_s(params: dict, x: float) -> float:
    p = make_problem(params)
    return lib().dse_ref_map(ctypes.byref(p), float(x))


def basis(params: dict, x: float) -> np.ndarray:
    p = make_problem(params)
    phi = np.empty(max(orders(params)))
    _chk(lib().dse_ref_basis(ctypes.byref(p), float(x), _ptr(phi)), "basis")
    return phi


def dressing(params: dict, c, x):
    p = make_problem(params)
    c = _f64(c); x = _f64(np.atleast_1d(x))
    lG = np.empty(x.size); lZ = np.empty(x.size)
    _chk(lib().dse_ref_dressing(ctypes.byref(p), _ptr(c), x.size, _ptr(x), _ptr(lG), _ptr(lZ)), "dressing")
    return lG, lZ


def kernels(x: float, y: float, theta: float):
    M = ctypes.c_double(); Q = ctypes.c_double(); z = ctypes.c_double()
    _chk(lib().dse_ref_kernels(float(x), float(y), float(theta), ctypes.byref(M), ctypes.byref(Q),
                               ctypes.byref(z)), "kernels")
    return M.value, Q.value, z.value


def self_energy(params: dict, c, x: float, grad: bool = False):
    p = make_problem(params)
    c = _f64(c)
    PiG = ctypes.c_double(); PiZ = ctypes.c_double()
    n = n_unknowns(params)
    dG = np.empty(n) if grad else None
    dZ = np.empty(n) if grad else None
    _chk(lib().dse_ref_self_energy(ctypes.byref(p), _ptr(c), float(x), ctypes.byref(PiG), ctypes.byref(PiZ),
                                   _ptr(dG) if grad else None, _ptr(dZ) if grad else None), "self_energy")
    if grad:
        return PiG.value, PiZ.value, dG, dZ
    return PiG.value, PiZ.value


def residual(params: dict, c) -> np.ndarray:
    p = make_problem(params)
    c = _f64(c)
    F = np.empty(n_unknowns(params))
    _chk(lib().dse_ref_residual(ctypes.byref(p), _ptr(c), _ptr(F)), "residual")
    return F


def newton_matrix(params: dict, c):
    p = make_problem(params)
    c = _f64(c)
    n = n_unknowns(params)
    J = np.empty((n, n)); F = np.empty(n)
    _chk(lib().dse_ref_newton_matrix(ctypes.byref(p), _ptr(c), _ptr(J), _ptr(F)), "newton_matrix")
    return J, F


def newton_matrix_magnitudes(params: dict, c):
    """(A, AF): sums of |summands| of every entry of J and F (rounding scale)."""
    p = make_problem(params)
    c = _f64(c)
    n = n_unknowns(params)
    A = np.empty((n, n)); AF = np.empty(n)
    _chk(lib().dse_ref_newton_matrix_magnitudes(ctypes.byref(p), _ptr(c), _ptr(A), _ptr(AF)),
         "newton_matrix_magnitudes")
    return A, AF


def param_derivatives(params: dict, c) -> np.ndarray:
    """dF/d(g2nc, ginv_G, zinv_Z): n x 3."""
    p = make_problem(params)
    c = _f64(c)
    dF = np.empty((n_unknowns(params), 3))
    _chk(lib().dse_ref_param_derivatives(ctypes.byref(p), _ptr(c), _ptr(dF)), "param_derivatives")
    return dF


def lu_solve(A, b) -> np.ndarray:
    A = _f64(A); b = _f64(b)
    x = np.empty(b.size)
    _chk(lib().dse_ref_lu_solve(b.size, _ptr(A), _ptr(b), _ptr(x)), "lu_solve")
    return x


def newton_step(params: dict, c, rho: float = 1.0):
    """Return (new coefficients, stats = [||F||inf, scaled ||F||inf, ||Delta||inf])."""
    p = make_problem(params)
    c = _f64(c).copy()
    stats = np.empty(3)
    _chk(lib().dse_ref_newton_step(ctypes.byref(p), _ptr(c), float(rho), _ptr(stats)), "newton_step")
    return c, stats


def solve(params: dict, c0, tol: float = 1e-10, max_iter: int = 50, rho: float = 1.0):
    """Newton iteration until the scaled residual drops below tol.

    Returns (coefficients, iterations, history of stats)."""
    c = _f64(c0).copy()
    hist = []
    for it in range(max_iter):
        c_new, st = newton_step(params, c, rho)
        hist.append(st)
        if st[1] < tol:
            return c, it, hist
        c = c_new
    raise OracleError("Newton did not converge in %d iterations (last stats %s)" % (max_iter, hist[-1]))


def schwinger_nodes(params: dict, n: int):
    p = make_problem(params)
    pn = np.empty(n); wn = np.empty(n)
    _chk(lib().dse_ref_schwinger_nodes(ctypes.byref(p), n, _ptr(pn), _ptr(wn)), "schwinger_nodes")
    return pn, wn


def schwinger(params: dict, c, t, n_nodes: int) -> np.ndarray:
    p = make_problem(params)
    c = _f64(c); t = _f64(t)
    out = np.empty(t.size)
    _chk(lib().dse_ref_schwinger(ctypes.byref(p), _ptr(c), _ptr(t), t.size, n_nodes, _ptr(out)), "schwinger")
    return out


def num_threads() -> int:
    return lib().dse_ref_num_threads()
