"""Thin Python binding of the C ABI in ``include/fps.h`` (argument marshalling only).

Every function here forwards to ``libfps.so``; all arithmetic of the solve runs
in the library's CUDA kernels.  Tensors are passed as raw pointers: a CUDA
tensor is used in place (asynchronous on the plan's stream), a NumPy array or
CPU tensor is staged by the library itself.  If the library has not been built
the first call raises; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfps.so")

FPS_FP64 = 0
FPS_FP32_REFINE = 1
FPS_TIGHT_SPECTRUM = 0x100
_PRECISION = {"fp64": FPS_FP64, "fp32_refine": FPS_FP32_REFINE, "fp64_tight": FPS_FP64 | FPS_TIGHT_SPECTRUM,
              FPS_FP64: FPS_FP64, FPS_FP32_REFINE: FPS_FP32_REFINE}

STATUS = {
    0: "FPS_OK",
    -1: "FPS_ERR_INVALID_ARG",
    -2: "FPS_ERR_UNSUPPORTED",
    -3: "FPS_ERR_CUDA",
    -4: "FPS_ERR_NOT_CONVERGED",
    -5: "FPS_ERR_NONFINITE",
    -6: "FPS_ERR_TIMEOUT",
}


class FpsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class PlanInfo(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("dim", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("nrhs", ctypes.c_int),
        ("batch", ctypes.c_int64),
        ("J", ctypes.c_int),
        ("J_inner", ctypes.c_int),
        ("refine_rounds", ctypes.c_int),
        ("last_residual", ctypes.c_double),
        ("tol", ctypes.c_double),
        ("device_bytes", ctypes.c_int64),
        ("kernel_launches", ctypes.c_int64),
        ("seg_len", ctypes.c_int),
        ("inner_iterations", ctypes.c_int64),
        ("chain_mode", ctypes.c_int),
    ]


_lock = threading.Lock()
_lib: Optional[ctypes.CDLL] = None

EXPORTED = [
    "fps_plan_create", "fps_plan_create_batched", "fps_plan_set_stream", "fps_poisson_square_solve",
    "fps_poisson_cube_solve", "fps_poisson_adjoint", "fps_plan_info", "fps_plan_shifts", "fps_plan_destroy",
    "fps_status_string", "fps_last_error", "fps_zolotarev_shifts", "fps_square_bands", "fps_build_arch",
    "fps_plan_set_instrument", "fps_plan_kernel_times", "fps_poisson_square_solve_noalloc",
    "fps_square_spectral_interval", "fps_legendre_to_ctilde", "fps_solution_to_legendre", "fps_plan_pass_times",
    "fps_probe_fma_rate", "fps_plan_create_rect", "fps_poisson_dirichlet_solve", "fps_poisson_dirichlet_adjoint",
    "fps_plan_create_cylinder", "fps_poisson_cylinder_solve", "fps_cylinder_mode_interval", "fps_cylinder_operators",
]


def lib() -> ctypes.CDLL:
    """Load ``libfps.so`` (built by ``build_ext.build()``); raise if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise FpsError(-3, f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
        L.fps_plan_create.argtypes = [ctypes.POINTER(vp), i64, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                      ctypes.c_int, vp]
        L.fps_plan_create_batched.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(i64), i64, ctypes.c_int,
                                              ctypes.c_double, ctypes.c_int, vp]
        L.fps_plan_set_stream.argtypes = [vp, vp]
        L.fps_poisson_square_solve.argtypes = [vp, vp, vp]
        L.fps_poisson_cube_solve.argtypes = [vp, vp, vp]
        L.fps_poisson_adjoint.argtypes = [vp, vp, vp]
        L.fps_plan_info.argtypes = [vp, ctypes.POINTER(PlanInfo)]
        L.fps_plan_shifts.argtypes = [vp, i64, dp, ctypes.c_int]
        L.fps_plan_destroy.argtypes = [vp]
        L.fps_plan_destroy.restype = None
        L.fps_status_string.argtypes = [ctypes.c_int]
        L.fps_status_string.restype = ctypes.c_char_p
        L.fps_last_error.restype = ctypes.c_char_p
        L.fps_zolotarev_shifts.argtypes = [ctypes.c_double] * 5 + [ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp,
                                                                   dp, ctypes.c_int]
        L.fps_square_bands.argtypes = [i64, dp, dp]
        L.fps_plan_set_instrument.argtypes = [vp, ctypes.c_int]
        L.fps_plan_kernel_times.argtypes = [vp, ctypes.POINTER(ctypes.c_int), dp, dp]
        L.fps_plan_pass_times.argtypes = [vp, dp, dp]
        L.fps_probe_fma_rate.argtypes = [ctypes.c_int, dp]
        L.fps_plan_create_rect.argtypes = [ctypes.POINTER(vp), i64, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int, ctypes.c_int, vp]
        L.fps_poisson_square_solve_noalloc.argtypes = [i64, ctypes.c_double, vp, vp, vp]
        L.fps_square_spectral_interval.argtypes = [i64, ctypes.c_int, dp, dp]
        L.fps_legendre_to_ctilde.argtypes = [i64, vp, vp, vp]
        L.fps_solution_to_legendre.argtypes = [i64, vp, vp, vp]
        L.fps_poisson_dirichlet_solve.argtypes = [vp, vp, vp, vp]
        L.fps_poisson_dirichlet_adjoint.argtypes = [vp, vp, vp, vp]
        L.fps_plan_create_cylinder.argtypes = [ctypes.POINTER(vp), i64, i64, i64, ctypes.c_double, ctypes.c_int, vp]
        L.fps_poisson_cylinder_solve.argtypes = [vp, vp, vp]
        L.fps_cylinder_mode_interval.argtypes = [i64, i64, dp, dp]
        L.fps_cylinder_operators.argtypes = [i64, i64, dp, dp]
        _lib = L
        return L


def _check(status: int) -> int:
    if status < 0:
        raise FpsError(status, lib().fps_last_error().decode())
    return status


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ptr(x) -> int:
    """Raw pointer of a contiguous FP64 tensor/array (marshalling only)."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags.c_contiguous:
            raise FpsError(-1, "arrays must be contiguous float64")
        return x.ctypes.data
    import torch

    if isinstance(x, torch.Tensor):
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise FpsError(-1, "tensors must be contiguous float64")
        return x.data_ptr()
    raise FpsError(-1, f"unsupported buffer type {type(x)}")


def _current_stream() -> int:
    try:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:  # pragma: no cover
        pass
    return 0


class Plan:
    """Owning handle of an ``fps_plan``."""

    def __init__(self, handle: int, n: int, dim: int, nrhs: int, batch_ns=None):
        self._h = ctypes.c_void_p(handle)
        self.n, self.dim, self.nrhs = n, dim, nrhs
        self.batch_ns = batch_ns

    @property
    def handle(self) -> ctypes.c_void_p:
        if not self._h:
            raise FpsError(-1, "plan already destroyed")
        return self._h

    def info(self) -> dict:
        return plan_info(self)

    def destroy(self) -> None:
        plan_destroy(self)

    def __del__(self):  # pragma: no cover - best effort
        try:
            if self._h:
                plan_destroy(self)
        except Exception:
            pass

    def shape(self):
        if self.batch_ns is not None:
            return (int(sum(self.nrhs * int(m) ** 2 for m in self.batch_ns)),)
        if self.dim == 2:
            return (self.nrhs, self.n, self.n) if self.nrhs > 1 else (self.n, self.n)
        return (self.nrhs, self.n, self.n, self.n) if self.nrhs > 1 else (self.n, self.n, self.n)


# ---------------------------------------------------------------- the C ABI, by name
def plan_create(n: int, dim: int = 2, tol: float = 1e-13, precision="fp64", nrhs: int = 1,
                stream: Optional[int] = None) -> Plan:
    h = ctypes.c_void_p()
    s = _current_stream() if stream is None else int(stream)
    _check(lib().fps_plan_create(ctypes.byref(h), int(n), int(dim), float(tol), _PRECISION[precision], int(nrhs),
                                 ctypes.c_void_p(s)))
    return Plan(h.value, int(n), int(dim), int(nrhs))


def plan_create_rect(n: int, width: float, height: float, tol: float = 1e-13, precision="fp64", nrhs: int = 1,
                     stream: Optional[int] = None) -> Plan:
    """Plan on a width x height rectangle (homogeneous Dirichlet); solve with
    poisson_square_solve."""
    h = ctypes.c_void_p()
    s = _current_stream() if stream is None else int(stream)
    _check(lib().fps_plan_create_rect(ctypes.byref(h), int(n), float(width), float(height), float(tol),
                                      _PRECISION[precision], int(nrhs), ctypes.c_void_p(s)))
    return Plan(h.value, int(n), 2, int(nrhs))


def plan_create_batched(ns, nrhs: int = 1, tol: float = 1e-10, precision="fp32_refine",
                        stream: Optional[int] = None) -> Plan:
    arr = np.ascontiguousarray(np.asarray(ns, dtype=np.int64))
    h = ctypes.c_void_p()
    s = _current_stream() if stream is None else int(stream)
    _check(lib().fps_plan_create_batched(ctypes.byref(h), arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                         len(arr), int(nrhs), float(tol), _PRECISION[precision],
                                         ctypes.c_void_p(s)))
    return Plan(h.value, int(arr.max()), 2, int(nrhs), batch_ns=arr)


def plan_set_stream(plan: Plan, stream: int) -> None:
    _check(lib().fps_plan_set_stream(plan.handle, ctypes.c_void_p(int(stream))))


def _out_like(F, X):
    if X is not None:
        return X
    if isinstance(F, np.ndarray):
        return np.empty_like(F)
    import torch

    return torch.empty_like(F)


def _numel(x) -> int:
    return int(x.size) if isinstance(x, np.ndarray) else int(x.numel())


def _check_plan_buffers(plan: Plan, F, X) -> None:
    """F must have the plan's shape (or be the packed 1-D array of that many
    elements) and X as many elements: the library reads and writes exactly that."""
    want = tuple(plan.shape())
    count = int(np.prod(want))
    shape = tuple(F.shape)
    if not (shape == want or (len(shape) == 1 and shape[0] == count)):
        raise FpsError(-1, f"input has shape {shape}; the plan expects {want}")
    if _numel(X) != count:
        raise FpsError(-1, f"output has {_numel(X)} elements; the plan writes {count}")


def poisson_square_solve(plan: Plan, F, X=None):
    X = _out_like(F, X)
    _check_plan_buffers(plan, F, X)
    _check(lib().fps_poisson_square_solve(plan.handle, ctypes.c_void_p(_ptr(F)), ctypes.c_void_p(_ptr(X))))
    return X


def poisson_cube_solve(plan: Plan, F, X=None):
    X = _out_like(F, X)
    _check_plan_buffers(plan, F, X)
    _check(lib().fps_poisson_cube_solve(plan.handle, ctypes.c_void_p(_ptr(F)), ctypes.c_void_p(_ptr(X))))
    return X


def poisson_adjoint(plan: Plan, dLdX, dLdF=None):
    dLdF = _out_like(dLdX, dLdF)
    _check_plan_buffers(plan, dLdX, dLdF)
    _check(lib().fps_poisson_adjoint(plan.handle, ctypes.c_void_p(_ptr(dLdX)), ctypes.c_void_p(_ptr(dLdF))))
    return dLdF


def plan_info(plan: Plan) -> dict:
    info = PlanInfo()
    _check(lib().fps_plan_info(plan.handle, ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in PlanInfo._fields_}


def plan_shifts(plan: Plan, problem: int = 0) -> np.ndarray:
    cap = 4096
    q = np.zeros(cap)
    J = _check(lib().fps_plan_shifts(plan.handle, int(problem), _dp(q), cap))
    return q[:J].copy()


def plan_set_instrument(plan: Plan, on: bool = True) -> None:
    _check(lib().fps_plan_set_instrument(plan.handle, 1 if on else 0))


def plan_kernel_times(plan: Plan) -> dict:
    """Dominant-kernel launches of the last solve: count, summed ms, algorithmic bytes."""
    c = ctypes.c_int()
    ms = ctypes.c_double()
    by = ctypes.c_double()
    _check(lib().fps_plan_kernel_times(plan.handle, ctypes.byref(c), ctypes.byref(ms), ctypes.byref(by)))
    rm, cm = ctypes.c_double(), ctypes.c_double()
    _check(lib().fps_plan_pass_times(plan.handle, ctypes.byref(rm), ctypes.byref(cm)))
    return {"count": c.value, "total_ms": ms.value, "alg_bytes": by.value, "row_ms": rm.value, "col_ms": cm.value}


def plan_destroy(plan: Plan) -> None:
    if plan._h:
        lib().fps_plan_destroy(plan._h)
        plan._h = ctypes.c_void_p()


def legendre_to_ctilde(G, F=None, stream: Optional[int] = None):
    """C~ coefficients F (n x n) of sum G_ab P_a(y) P_b(x); CUDA float64 tensors."""
    import torch

    n = int(G.shape[-1])
    if tuple(G.shape) != (n, n):
        raise FpsError(-1, f"G has shape {tuple(G.shape)}; expected a square matrix")
    F = torch.empty_like(G) if F is None else F
    if tuple(F.shape) != (n, n):
        raise FpsError(-1, f"F has shape {tuple(F.shape)}; expected {(n, n)}")
    s = _current_stream() if stream is None else int(stream)
    _check(lib().fps_legendre_to_ctilde(n, ctypes.c_void_p(_ptr(G)), ctypes.c_void_p(_ptr(F)), ctypes.c_void_p(s)))
    return F


def solution_to_legendre(X, U=None, stream: Optional[int] = None):
    """Legendre coefficients U ((n+2) x (n+2)) of u = (1-x^2)(1-y^2) sum X_ij C~_i(y) C~_j(x)."""
    import torch

    n = int(X.shape[-1])
    if tuple(X.shape) != (n, n):
        raise FpsError(-1, f"X has shape {tuple(X.shape)}; expected a square matrix")
    U = torch.empty((n + 2, n + 2), dtype=X.dtype, device=X.device) if U is None else U
    if tuple(U.shape) != (n + 2, n + 2):
        raise FpsError(-1, f"U has shape {tuple(U.shape)}; expected {(n + 2, n + 2)}")
    s = _current_stream() if stream is None else int(stream)
    _check(lib().fps_solution_to_legendre(n, ctypes.c_void_p(_ptr(X)), ctypes.c_void_p(_ptr(U)), ctypes.c_void_p(s)))
    return U


def _dirichlet_shapes(plan: Plan):
    """Shapes of (G or dL/dG, bc or dL/dbc, U or dL/dU) for a square / rectangle plan."""
    if plan.dim != 2 or plan.batch_ns is not None:
        raise FpsError(-1, "nonhomogeneous Dirichlet solves need a single square or rectangle plan")
    n, m = plan.n, plan.n + 2
    lead = (plan.nrhs,) if plan.nrhs > 1 else ()
    return lead + (n, n), lead + (4, m), lead + (m, m)


def _need_shape(x, shape, name):
    if tuple(x.shape) != tuple(shape):
        raise FpsError(-1, f"{name} has shape {tuple(x.shape)}; the plan expects {tuple(shape)}")


def poisson_dirichlet_solve(plan: Plan, G, bc, U=None):
    """Legendre coefficients U ((n+2) x (n+2)) of the solution with Dirichlet traces bc
    ([g_W, g_E, g_S, g_N], each n+2 Legendre coefficients) and right-hand side G (n x n
    Legendre coefficients); CUDA float64 tensors, a leading nrhs axis when nrhs > 1."""
    import torch

    sg, sb, su = _dirichlet_shapes(plan)
    _need_shape(G, sg, "G")
    _need_shape(bc, sb, "bc")
    U = torch.empty(su, dtype=G.dtype, device=G.device) if U is None else U
    _need_shape(U, su, "U")
    _check(lib().fps_poisson_dirichlet_solve(plan.handle, ctypes.c_void_p(_ptr(G)), ctypes.c_void_p(_ptr(bc)),
                                             ctypes.c_void_p(_ptr(U))))
    return U


def poisson_dirichlet_adjoint(plan: Plan, dLdU, dLdG=None, dLdbc=None):
    """(dL/dG, dL/dbc) from dL/dU through poisson_dirichlet_solve."""
    import torch

    sg, sb, su = _dirichlet_shapes(plan)
    _need_shape(dLdU, su, "dLdU")
    dLdG = torch.empty(sg, dtype=dLdU.dtype, device=dLdU.device) if dLdG is None else dLdG
    dLdbc = torch.empty(sb, dtype=dLdU.dtype, device=dLdU.device) if dLdbc is None else dLdbc
    _need_shape(dLdG, sg, "dLdG")
    _need_shape(dLdbc, sb, "dLdbc")
    _check(lib().fps_poisson_dirichlet_adjoint(plan.handle, ctypes.c_void_p(_ptr(dLdU)), ctypes.c_void_p(_ptr(dLdG)),
                                               ctypes.c_void_p(_ptr(dLdbc))))
    return dLdG, dLdbc


class CylinderPlan(Plan):
    """Plan over the cylinder's Fourier modes kmin .. kmax (Sec. 4.1, Case 1)."""

    def __init__(self, handle: int, n: int, kmin: int, kmax: int, nrhs: int):
        super().__init__(handle, n, 3, nrhs)
        self.kmin, self.kmax = kmin, kmax

    def shape(self):
        return (self.kmax - self.kmin + 1, self.nrhs, self.n, self.n)


def plan_create_cylinder(n: int, kmin: int, kmax: int, tol: float = 1e-13, nrhs: int = 1,
                         stream: Optional[int] = None) -> CylinderPlan:
    h = ctypes.c_void_p()
    s = _current_stream() if stream is None else int(stream)
    _check(lib().fps_plan_create_cylinder(ctypes.byref(h), int(n), int(kmin), int(kmax), float(tol), int(nrhs),
                                          ctypes.c_void_p(s)))
    return CylinderPlan(h.value, int(n), int(kmin), int(kmax), int(nrhs))


def poisson_cylinder_solve(plan: CylinderPlan, F, Y=None):
    """Y [modes][nrhs][n][n]: coefficients of w_k for every mode and right-hand side."""
    if not isinstance(plan, CylinderPlan):
        raise FpsError(-1, "not a cylinder plan")
    Y = _out_like(F, Y)
    _need_shape(F, plan.shape(), "F")
    _need_shape(Y, plan.shape(), "Y")
    _check(lib().fps_poisson_cylinder_solve(plan.handle, ctypes.c_void_p(_ptr(F)), ctypes.c_void_p(_ptr(Y))))
    return Y


def cylinder_mode_interval(n: int, k: int):
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().fps_cylinder_mode_interval(int(n), int(k), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def cylinder_operators(n: int, k: int = 2):
    L1 = np.zeros((n, n))
    Q = np.zeros((n, n))
    _check(lib().fps_cylinder_operators(int(n), int(k), _dp(L1), _dp(Q)))
    return L1, Q


def poisson_square_solve_noalloc(F, X, tol: float = 1e-13, stream: Optional[int] = None) -> int:
    """FP64 square solve for n <= 256 that allocates nothing (see fps.h); F and X are
    caller-allocated n x n CUDA tensors on one device.  Returns the status code (0 = ok);
    a malformed shape raises before the library is called."""
    if len(F.shape) != 2 or F.shape[0] != F.shape[1] or tuple(X.shape) != tuple(F.shape):
        raise FpsError(-1, f"F and X must both be n x n (got {tuple(F.shape)} and {tuple(X.shape)})")
    if getattr(F, "device", None) != getattr(X, "device", None):
        raise FpsError(-1, "F and X must be on the same device")
    s = _current_stream() if stream is None else int(stream)
    return int(lib().fps_poisson_square_solve_noalloc(int(F.shape[-1]), float(tol), ctypes.c_void_p(_ptr(F)),
                                                      ctypes.c_void_p(_ptr(X)), ctypes.c_void_p(s)))


def probe_fma_rate(precision="fp64") -> float:
    """Measured FMAs per second of the current device (FP64 or FP32)."""
    r = ctypes.c_double()
    _check(lib().fps_probe_fma_rate(_PRECISION[precision], ctypes.byref(r)))
    return r.value


def zolotarev_shifts(a: float, b: float, c: float, d: float, tol: float, J: int = 0):
    Jo = ctypes.c_int()
    _check(lib().fps_zolotarev_shifts(a, b, c, d, tol, int(J), ctypes.byref(Jo), None, None, 0))
    p, q = np.zeros(Jo.value), np.zeros(Jo.value)
    _check(lib().fps_zolotarev_shifts(a, b, c, d, tol, int(J), ctypes.byref(Jo), _dp(p), _dp(q), Jo.value))
    return p, q


def square_spectral_interval(n: int, tight: bool = False):
    """(lo, hi) with sigma(A~) in [-hi, -lo]: Lemma B.2, or tight bounds by bisection."""
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _check(lib().fps_square_spectral_interval(int(n), 1 if tight else 0, ctypes.byref(lo), ctypes.byref(hi)))
    return lo.value, hi.value


def square_bands(n: int):
    d = np.zeros(n)
    e = np.zeros(max(n - 2, 1))
    _check(lib().fps_square_bands(int(n), _dp(d), _dp(e)))
    return d, e[: max(n - 2, 0)]


def status_string(status: int) -> str:
    return lib().fps_status_string(int(status)).decode()
