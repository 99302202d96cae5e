"""ctypes binding of include/dse.h (argument marshalling only).

Device buffers are torch tensors (CUDA, float64, contiguous); the plan follows
torch's current CUDA stream.  There is no CPU fallback: if the CUDA library is
missing the import of the binding's entry points fails with an error."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

DSE_OK = 0
DSE_ERR_ARG = -1
DSE_ERR_NONFINITE = -2
DSE_ERR_SINGULAR = -3
DSE_ERR_CUDA = -4
DSE_ERR_UNSUPPORTED = -5
DSE_ERR_NOT_CONVERGED = -6
DSE_MAX_CHEB = 256

EXPORTS = ["dse_plan_create", "dse_plan_destroy", "dse_plan_set_stream", "dse_plan_status", "dse_quadrature",
           "dse_dressing", "dse_residual", "dse_newton_matrix", "dse_newton_step", "dse_solve", "dse_schwinger",
           "dse_plan_profile", "dse_plan_counters", "dse_residual_static", "dse_status_string",
           "dse_plan_set_couplings", "dse_vjp", "dse_param_derivatives", "dse_adjoint_solve", "dse_dressing_vjp",
           "dse_batch_create", "dse_batch_destroy", "dse_batch_set_stream", "dse_batch_offsets", "dse_batch_tune",
           "dse_batch_newton_matrix", "dse_batch_solve", "dse_batch_counters", "dse_newton_matrix_fd",
           "dse_batch_residual", "dse_plan_solver_counters", "dse_alu_peak"]

# pipes of dse_alu_peak (include/dse_peaks.h)
DSE_PEAK_FP64_FMA = 0
DSE_PEAK_FP32_FMA = 1
DSE_PEAK_MUFU_EX2 = 2
DSE_PEAK_MUFU_LG2 = 3
DSE_PEAK_FP64_DMMA = 4
DSE_PEAK_FP32X2_FMA = 5


class DseError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__("%s: %s (status %d)" % (what, status_string(code), code))


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

    @classmethod
    def from_params(cls, params: dict) -> "Problem":
        p = cls()
        for name, _ in cls._fields_:
            setattr(p, name, params.get(name, 0) if name in ("n_cheb_G", "angular_mode") else params[name])
        return p


_lib = None
_VP = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load the CUDA library (raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError("dse CUDA library not built (%s); run __graft_entry__.build()" % path)
    L = ctypes.CDLL(path)
    PP = ctypes.POINTER(Problem)
    sig = {
        "dse_plan_create": [PP, _VP, ctypes.POINTER(_VP)],
        "dse_plan_destroy": [_VP],
        "dse_plan_set_stream": [_VP, _VP],
        "dse_plan_status": [_VP],
        "dse_quadrature": [_VP, _VP, _VP, _VP, _VP, _VP],
        "dse_dressing": [_VP, _VP, ctypes.c_int, _VP, _VP, _VP],
        "dse_residual": [_VP, _VP, _VP],
        "dse_newton_matrix": [_VP, _VP, _VP, _VP],
        "dse_newton_step": [_VP, _VP, ctypes.c_double, _D],
        "dse_solve": [_VP, _VP, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                      ctypes.POINTER(ctypes.c_int), _D],
        "dse_schwinger": [_VP, _VP, _VP, ctypes.c_int, ctypes.c_int, _VP],
        "dse_plan_profile": [_VP, ctypes.c_int],
        "dse_residual_static": [PP, _VP, _VP, _VP],
        "dse_plan_counters": [_VP, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_int),
                              ctypes.POINTER(ctypes.c_double)],
        "dse_plan_solver_counters": [_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
        "dse_plan_set_couplings": [_VP, ctypes.c_double, ctypes.c_double, ctypes.c_double],
        "dse_vjp": [_VP, _VP, _VP, _VP, _VP],
        "dse_param_derivatives": [_VP, _VP, _VP, _VP, _VP],
        "dse_adjoint_solve": [_VP, _VP, _VP, _VP, _D],
        "dse_dressing_vjp": [_VP, ctypes.c_int, _VP, _VP, _VP, _VP, _VP],
        "dse_batch_create": [PP, ctypes.c_int, _VP, ctypes.POINTER(_VP)],
        "dse_batch_destroy": [_VP],
        "dse_batch_set_stream": [_VP, _VP],
        "dse_batch_offsets": [_VP, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)],
        "dse_batch_tune": [_VP, _VP, ctypes.POINTER(ctypes.c_int), _D],
        "dse_batch_newton_matrix": [_VP, _VP, _VP, _VP],
        "dse_batch_residual": [_VP, _VP, _VP],
        "dse_newton_matrix_fd": [_VP, _VP, ctypes.c_double, _VP, _VP],
        "dse_batch_solve": [_VP, _VP, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _D],
        "dse_batch_counters": [_VP, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                               ctypes.POINTER(ctypes.c_int)],
        "dse_alu_peak": [ctypes.c_int, ctypes.c_double, _VP, _D, _D],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.dse_status_string.argtypes = [ctypes.c_int]
    L.dse_status_string.restype = ctypes.c_char_p
    _lib = L
    return L


def alu_peak(kind: int, target_ms: float = 100.0):
    """(operations per second, ms) of one arithmetic pipe on the current device,
    on torch's current stream (dse_alu_peak)."""
    import torch
    L = load()
    rate, ms = ctypes.c_double(), ctypes.c_double()
    _check(L.dse_alu_peak(int(kind), float(target_ms), _VP(torch.cuda.current_stream().cuda_stream),
                          ctypes.byref(rate), ctypes.byref(ms)), "dse_alu_peak")
    return rate.value, ms.value


def status_string(code: int) -> str:
    try:
        return load().dse_status_string(int(code)).decode()
    except Exception:  # library not loadable: plain code
        return "status %d" % code


def _check(code: int, what: str) -> None:
    if code != DSE_OK:
        raise DseError(code, what)


def _dev_ptr(t, n: int, name: str):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % name)
    if t.device.type != "cuda" or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError("%s must be a contiguous float64 CUDA tensor" % name)
    if t.numel() < n:
        raise ValueError("%s has %d elements, needs %d" % (name, t.numel(), n))
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Plan:
    """A dse_plan for one problem (workspace and quadrature rules on the current device)."""

    def __init__(self, params: dict):
        import torch
        self._L = load()
        self.params = dict(params)
        self.NZ = int(params["n_cheb"])
        self.NG = int(params.get("n_cheb_G", 0) or 0) or self.NZ
        self.N = max(self.NZ, self.NG)
        self.n = self.NZ + self.NG
        self.n_collocation = self.N if self.NZ == self.NG else self.n
        self.n_radial = int(params["n_radial"])
        self.n_angular = int(params["n_angular"])
        self.device = torch.device("cuda", torch.cuda.current_device())
        prob = Problem.from_params(self.params)
        h = _VP()
        _check(self._L.dse_plan_create(ctypes.byref(prob), _stream_ptr(), ctypes.byref(h)), "dse_plan_create")
        self._h = h

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._L.dse_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _sync_stream(self) -> None:
        self._L.dse_plan_set_stream(self._h, _stream_ptr())

    def _new(self, *shape):
        import torch
        return torch.empty(*shape, dtype=torch.float64, device=self.device)

    def quadrature(self):
        nrad = self.n_radial * (3 if self.params.get("radial_mode", 0) == 1 else 1)
        y, W, th, wt, x = (self._new(nrad), self._new(nrad), self._new(self.n_angular),
                           self._new(self.n_angular), self._new(self.n_collocation))
        self._sync_stream()
        _check(self._L.dse_quadrature(self._h, *[ctypes.c_void_p(t.data_ptr()) for t in (y, W, th, wt, x)]),
               "dse_quadrature")
        return y, W, th, wt, x

    def dressing(self, coeffs, x):
        n = x.numel()
        lG, lZ = self._new(n), self._new(n)
        self._sync_stream()
        _check(self._L.dse_dressing(self._h, _dev_ptr(coeffs, self.n, "coeffs"), n, _dev_ptr(x, n, "x"),
                                    ctypes.c_void_p(lG.data_ptr()), ctypes.c_void_p(lZ.data_ptr())), "dse_dressing")
        return lG, lZ

    def residual(self, coeffs, out=None):
        F = out if out is not None else self._new(self.n)
        self._sync_stream()
        _check(self._L.dse_residual(self._h, _dev_ptr(coeffs, self.n, "coeffs"), _dev_ptr(F, self.n, "F")),
               "dse_residual")
        return F

    def newton_matrix(self, coeffs, J=None, F=None):
        n = self.n
        J = J if J is not None else self._new(n, n)
        F = F if F is not None else self._new(n)
        self._sync_stream()
        _check(self._L.dse_newton_matrix(self._h, _dev_ptr(coeffs, n, "coeffs"), _dev_ptr(J, n * n, "J"),
                                         _dev_ptr(F, n, "F")), "dse_newton_matrix")
        return J, F

    def newton_matrix_fd(self, coeffs, rel_step: float = 1e-5, J=None, F=None):
        """The paper's central-difference Newton matrix (batched perturbed residuals)."""
        n = self.n
        J = J if J is not None else self._new(n, n)
        self._sync_stream()
        _check(self._L.dse_newton_matrix_fd(self._h, _dev_ptr(coeffs, n, "coeffs"), float(rel_step),
                                            _dev_ptr(J, n * n, "J"), _dev_ptr(F, n, "F") if F is not None else None),
               "dse_newton_matrix_fd")
        return J

    def newton_step(self, coeffs, rho: float = 1.0):
        """In-place Newton step; returns (||F||inf, scaled ||F||inf, ||Delta||inf) on entry
        and the number of FP64 refinement sweeps (-1: FP64 LU)."""
        st = (ctypes.c_double * 4)()
        self._sync_stream()
        _check(self._L.dse_newton_step(self._h, _dev_ptr(coeffs, self.n, "coeffs"), float(rho),
                                       ctypes.cast(st, _D)), "dse_newton_step")
        return tuple(st)

    def solve(self, coeffs, tol: float = 1e-10, max_iter: int = 50, rho_relax: float = 1.0, n_relax: int = 0):
        """In-place Newton iteration; returns (iterations, stats of the last step)."""
        st = (ctypes.c_double * 3)()
        it = ctypes.c_int(0)
        self._sync_stream()
        _check(self._L.dse_solve(self._h, _dev_ptr(coeffs, self.n, "coeffs"), float(tol), int(max_iter),
                                 float(rho_relax), int(n_relax), ctypes.byref(it), ctypes.cast(st, _D)), "dse_solve")
        return it.value, tuple(st)

    def schwinger(self, coeffs, t, n_nodes: int, out=None):
        n_t = t.numel()
        out = out if out is not None else self._new(n_t)
        self._sync_stream()
        _check(self._L.dse_schwinger(self._h, _dev_ptr(coeffs, self.n, "coeffs"), _dev_ptr(t, n_t, "t"), n_t,
                                     int(n_nodes), _dev_ptr(out, n_t, "delta")), "dse_schwinger")
        return out

    def set_couplings(self, g2nc: float, ginv_G: float, zinv_Z: float) -> None:
        self._sync_stream()
        _check(self._L.dse_plan_set_couplings(self._h, float(g2nc), float(ginv_G), float(zinv_Z)),
               "dse_plan_set_couplings")
        self.params.update(g2nc=float(g2nc), ginv_G=float(ginv_G), zinv_Z=float(zinv_Z))

    def vjp(self, coeffs, v, out=None, F=None):
        """v^T dF/dc (2N); F (optional tensor) receives the residual."""
        n = self.n
        out = out if out is not None else self._new(n)
        self._sync_stream()
        _check(self._L.dse_vjp(self._h, _dev_ptr(coeffs, n, "coeffs"), _dev_ptr(v, n, "v"), _dev_ptr(out, n, "out"),
                               _dev_ptr(F, n, "F") if F is not None else None), "dse_vjp")
        return out

    def param_derivatives(self, coeffs):
        """dF/d(g2nc, ginv_G, zinv_Z): 2N x 3."""
        n = self.n
        dF = self._new(n, 3)
        self._sync_stream()
        _check(self._L.dse_param_derivatives(self._h, _dev_ptr(coeffs, n, "coeffs"), _dev_ptr(dF, 3 * n, "dF"),
                                             None, None), "dse_param_derivatives")
        return dF

    def param_vjp(self, coeffs, v, out=None):
        """v^T dF/d(g2nc, ginv_G, zinv_Z): 3."""
        n = self.n
        out = out if out is not None else self._new(3)
        self._sync_stream()
        _check(self._L.dse_param_derivatives(self._h, _dev_ptr(coeffs, n, "coeffs"), None, _dev_ptr(v, n, "v"),
                                             _dev_ptr(out, 3, "vdF")), "dse_param_derivatives")
        return out

    def adjoint_solve(self, coeffs, g, out=None):
        """lambda with J(c)^T lambda = g; returns (lambda, stats)."""
        n = self.n
        out = out if out is not None else self._new(n)
        st = (ctypes.c_double * 4)()
        self._sync_stream()
        _check(self._L.dse_adjoint_solve(self._h, _dev_ptr(coeffs, n, "coeffs"), _dev_ptr(g, n, "g"),
                                         _dev_ptr(out, n, "lambda"), ctypes.cast(st, _D)), "dse_adjoint_solve")
        return out, tuple(st)

    def dressing_vjp(self, x, gG, gZ, out=None, out_g2nc=None):
        """(sum gZ dlnZ/da, sum gG dlnG/db) as one 2N vector, and optionally d/d g2nc into out_g2nc (1)."""
        m = x.numel()
        n = self.n
        out = out if out is not None else self._new(n)
        self._sync_stream()
        _check(self._L.dse_dressing_vjp(self._h, m, _dev_ptr(x, m, "x"), _dev_ptr(gG, m, "gG"), _dev_ptr(gZ, m, "gZ"),
                                        _dev_ptr(out, n, "out"),
                                        _dev_ptr(out_g2nc, 1, "out_g2nc") if out_g2nc is not None else None),
               "dse_dressing_vjp")
        return out

    def status(self) -> int:
        return self._L.dse_plan_status(self._h)

    def profile(self, enable: bool = True) -> None:
        _check(self._L.dse_plan_profile(self._h, int(bool(enable))), "dse_plan_profile")

    def counters(self):
        """(kernel launches since creation, timed hot-kernel launches, their device ms)."""
        n = ctypes.c_longlong(0)
        k = ctypes.c_int(0)
        ms = ctypes.c_double(0.0)
        _check(self._L.dse_plan_counters(self._h, ctypes.byref(n), ctypes.byref(k), ctypes.byref(ms)),
               "dse_plan_counters")
        return n.value, k.value, ms.value

    def solver_counters(self):
        """(Newton steps that eliminated, steps solved with a kept inverse) since creation (n <= 128)."""
        e = ctypes.c_int(0)
        r = ctypes.c_int(0)
        _check(self._L.dse_plan_solver_counters(self._h, ctypes.byref(e), ctypes.byref(r)),
               "dse_plan_solver_counters")
        return e.value, r.value


class Batch:
    """A dse_batch: independent problems solved together (coefficients concatenated
    in problem order; offsets() gives the slices)."""

    def __init__(self, problems):
        import torch
        self._L = load()
        self.problems = [dict(p) for p in problems]
        self.nb = len(self.problems)
        arr = (Problem * self.nb)(*[Problem.from_params(p) for p in self.problems])
        h = _VP()
        _check(self._L.dse_batch_create(arr, self.nb, _stream_ptr(), ctypes.byref(h)), "dse_batch_create")
        self._h = h
        self.device = torch.device("cuda", torch.cuda.current_device())
        off = (ctypes.c_longlong * (self.nb + 1))()
        moff = (ctypes.c_longlong * (self.nb + 1))()
        _check(self._L.dse_batch_offsets(self._h, off, moff), "dse_batch_offsets")
        self.offsets = [int(v) for v in off]
        self.matrix_offsets = [int(v) for v in moff]
        self.n_total = self.offsets[-1]

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._L.dse_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _sync_stream(self) -> None:
        self._L.dse_batch_set_stream(self._h, _stream_ptr())

    def split(self, t):
        """Per-problem views of a concatenated coefficient (or residual) vector."""
        return [t[self.offsets[b]:self.offsets[b + 1]] for b in range(self.nb)]

    def tune(self, coeffs):
        """Pick the radial nodes per work item by timing; returns (choice, ms per candidate)."""
        u = ctypes.c_int(0)
        ms = (ctypes.c_double * 5)()
        self._sync_stream()
        _check(self._L.dse_batch_tune(self._h, _dev_ptr(coeffs, self.n_total, "coeffs"), ctypes.byref(u),
                                      ctypes.cast(ms, _D)), "dse_batch_tune")
        return u.value, list(ms)

    def residual(self, coeffs):
        """Concatenated residuals."""
        import torch
        F = torch.empty(self.n_total, dtype=torch.float64, device=self.device)
        self._sync_stream()
        _check(self._L.dse_batch_residual(self._h, _dev_ptr(coeffs, self.n_total, "coeffs"),
                                          _dev_ptr(F, self.n_total, "F")), "dse_batch_residual")
        return F

    def newton_matrix(self, coeffs):
        """(J, F): concatenated Newton matrices (flat) and residuals."""
        import torch
        J = torch.empty(self.matrix_offsets[-1], dtype=torch.float64, device=self.device)
        F = torch.empty(self.n_total, dtype=torch.float64, device=self.device)
        self._sync_stream()
        _check(self._L.dse_batch_newton_matrix(self._h, _dev_ptr(coeffs, self.n_total, "coeffs"),
                                               _dev_ptr(J, J.numel(), "J"), _dev_ptr(F, self.n_total, "F")),
               "dse_batch_newton_matrix")
        return J, F

    def matrices(self, J):
        """Per-problem n_b x n_b views of a concatenated matrix vector."""
        out = []
        for b in range(self.nb):
            n = self.offsets[b + 1] - self.offsets[b]
            out.append(J[self.matrix_offsets[b]:self.matrix_offsets[b + 1]].view(n, n))
        return out

    def solve(self, coeffs, tol: float = 1e-10, max_iter: int = 50, rho_relax: float = 1.0, n_relax: int = 0,
              check: bool = True):
        """In-place Newton iteration of every problem; returns (iterations, status codes, stats)."""
        it = (ctypes.c_int * self.nb)()
        st = (ctypes.c_int * self.nb)()
        stats = (ctypes.c_double * (3 * self.nb))()
        self._sync_stream()
        code = self._L.dse_batch_solve(self._h, _dev_ptr(coeffs, self.n_total, "coeffs"), float(tol), int(max_iter),
                                       float(rho_relax), int(n_relax), it, st, ctypes.cast(stats, _D))
        if code not in (DSE_OK, DSE_ERR_NOT_CONVERGED) or (check and code != DSE_OK):
            raise DseError(code, "dse_batch_solve")
        return list(it), list(st), [tuple(stats[3 * b:3 * b + 3]) for b in range(self.nb)]

    def counters(self):
        """(kernel launches, graph launches, radial nodes per work item)."""
        n = ctypes.c_longlong(0)
        g = ctypes.c_longlong(0)
        u = ctypes.c_int(0)
        _check(self._L.dse_batch_counters(self._h, ctypes.byref(n), ctypes.byref(g), ctypes.byref(u)),
               "dse_batch_counters")
        return n.value, g.value, u.value
