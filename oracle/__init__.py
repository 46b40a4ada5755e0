"""CPU oracle for the spectral Poisson ADI solver (arXiv 1710.11259).

TEST INFRASTRUCTURE ONLY.  This package is the independent checker of the GPU
library.  Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it; the GPU library never does, and the two
share no code (the seeded input generators live in a module of their own that
holds none of the method's arithmetic).

The arithmetic lives in ``fps_oracle.c`` (plain C, FP64; a long-double build
serves as a rounding check).  This module compiles it with gcc and exposes
numpy wrappers.  ``basis.py`` holds the quadrature tools for the normalised
ultraspherical basis used by the manufactured-solution pins.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fps_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS: dict[str, ctypes.CDLL] = {}

_VARIANTS = {
    "double": ("liboracle.so", []),
    "longdouble": ("liboracle_ld.so", ["-DORC_REAL=long double"]),
}


def _compile(variant: str) -> str:
    name, defs = _VARIANTS[variant]
    out = os.path.join(_BUILD, name)
    if os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", *defs, _SRC, "-lm"]
    tmp = out + f".tmp{os.getpid()}"
    # OpenMP only distributes independent right-hand sides; fall back to serial if absent.
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:] + ["-o", tmp], capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(base + ["-o", tmp], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"oracle build failed:\n{r.stderr}")
    os.replace(tmp, out)
    return out


def build() -> None:
    """Compile both oracle variants (double and long double)."""
    for v in _VARIANTS:
        _compile(v)


def _lib(variant: str = "double") -> ctypes.CDLL:
    with _LOCK:
        if variant not in _LIBS:
            lib = ctypes.CDLL(_compile(variant))
            c_dp = ctypes.POINTER(ctypes.c_double)
            lib.orc_M_bands.argtypes = [ctypes.c_long, c_dp, c_dp]
            lib.orc_square_bands.argtypes = [ctypes.c_long, c_dp, c_dp]
            lib.orc_adi_iterations.argtypes = [ctypes.c_double] * 5
            lib.orc_adi_iterations.restype = ctypes.c_int
            lib.orc_adi_shifts.argtypes = [ctypes.c_double] * 5 + [ctypes.c_int, c_dp, c_dp]
            lib.orc_adi_shifts.restype = ctypes.c_int
            lib.orc_adi_sylvester.argtypes = [ctypes.c_long, ctypes.c_int, c_dp, c_dp, c_dp, c_dp, c_dp,
                                              ctypes.c_int, c_dp, c_dp, c_dp]
            lib.orc_poisson_square.argtypes = [ctypes.c_long, ctypes.c_double, c_dp, c_dp]
            lib.orc_poisson_square.restype = ctypes.c_int
            lib.orc_poisson_square_tight.argtypes = [ctypes.c_long, ctypes.c_double, c_dp, c_dp]
            lib.orc_poisson_square_tight.restype = ctypes.c_int
            lib.orc_tight_interval.argtypes = [ctypes.c_long, c_dp, c_dp]
            lib.orc_poisson_rectangle.argtypes = [ctypes.c_long, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                  ctypes.c_int, c_dp, c_dp]
            lib.orc_poisson_rectangle.restype = ctypes.c_int
            lib.orc_poisson_square_partial.argtypes = [ctypes.c_long, ctypes.c_double, ctypes.c_int, c_dp, c_dp]
            lib.orc_poisson_square_partial.restype = ctypes.c_int
            lib.orc_poisson_cube.argtypes = [ctypes.c_long, ctypes.c_double, ctypes.c_double, ctypes.c_double, c_dp,
                                             c_dp, ctypes.POINTER(ctypes.c_int)]
            lib.orc_poisson_cube.restype = ctypes.c_long
            lib.orc_num_threads.restype = ctypes.c_int
            lib.orc_set_num_threads.argtypes = [ctypes.c_int]
            lib.orc_legendre_to_ctilde.argtypes = [ctypes.c_long, c_dp, c_dp]
            lib.orc_solution_to_legendre.argtypes = [ctypes.c_long, c_dp, c_dp]
            lib.orc_legendre_to_ctilde_adjoint.argtypes = [ctypes.c_long, c_dp, c_dp]
            lib.orc_solution_to_legendre_adjoint.argtypes = [ctypes.c_long, c_dp, c_dp]
            lib.orc_real_bytes.restype = ctypes.c_int
            _LIBS[variant] = lib
        return _LIBS[variant]


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# Section 3.2-3.3: the matrices of the discretisation
# --------------------------------------------------------------------------
def M_bands(n: int):
    """Diagonal (n) and second off-diagonal (n-2) of M, eq. (3.7)."""
    d = np.zeros(n)
    e = np.zeros(max(n - 2, 1))
    _lib().orc_M_bands(n, _ptr(d), _ptr(e))
    return d, e[: max(n - 2, 0)]


def square_bands(n: int):
    """Bands of A~ = D_s^{-1} D^{-1} M D_s, eq. (3.8)-(3.9): diagonal and (j, j+2)."""
    d = np.zeros(n)
    e = np.zeros(max(n - 2, 1))
    _lib().orc_square_bands(n, _ptr(d), _ptr(e))
    return d, e[: max(n - 2, 0)]


def square_interval(n: int):
    """Lemma B.2: sigma(A~) in [-1, -1/(30 n^4)], sigma(B~) = -sigma(A~)."""
    eps = 1.0 / (30.0 * float(n) ** 4)
    return -1.0, -eps, eps, 1.0


# --------------------------------------------------------------------------
# Theorem 2.1, eq. (2.9), Appendix A
# --------------------------------------------------------------------------
def adi_iterations(a: float, b: float, c: float, d: float, tol: float, variant: str = "double") -> int:
    return int(_lib(variant).orc_adi_iterations(a, b, c, d, tol))


def adi_shifts(a: float, b: float, c: float, d: float, tol: float, J: int | None = None,
               variant: str = "double"):
    """Zolotarev shifts (p, q) of (2.4); J from (2.9) unless given."""
    if J is None:
        J = adi_iterations(a, b, c, d, tol, variant)
    p = np.zeros(J)
    q = np.zeros(J)
    _lib(variant).orc_adi_shifts(a, b, c, d, tol, J, _ptr(p), _ptr(q))
    return p, q


def adi_sylvester(s: int, Ad, Ae, Bd, Be, F, p, q, variant: str = "double") -> np.ndarray:
    """Algorithm 2 on A X - X B = F with symmetric stride-s tridiagonal A, B."""
    F = _f64(F)
    n = F.shape[0]
    assert F.shape == (n, n)
    Ad, Bd = _f64(Ad), _f64(Bd)
    Ae = _f64(np.concatenate([np.asarray(Ae, dtype=np.float64), [0.0]]))
    Be = _f64(np.concatenate([np.asarray(Be, dtype=np.float64), [0.0]]))
    p, q = _f64(p), _f64(q)
    X = np.zeros_like(F)
    _lib(variant).orc_adi_sylvester(n, s, _ptr(Ad), _ptr(Ae), _ptr(Bd), _ptr(Be), _ptr(F), len(p), _ptr(p),
                                    _ptr(q), _ptr(X))
    return X


def poisson_square(F, tol: float = 1e-13, variant: str = "double", tight: bool = False) -> np.ndarray:
    """Solve M X D^T + D X M^T = F (eq. (3.6)) by Table 3.1 steps 2-3 (shifts from
    Lemma B.2's interval, or from ``tight_interval`` when ``tight``)."""
    F = _f64(F)
    n = F.shape[0]
    assert F.ndim == 2 and F.shape == (n, n)
    X = np.zeros_like(F)
    if tight:
        _lib(variant).orc_poisson_square_tight(n, tol, _ptr(F), _ptr(X))
    else:
        _lib(variant).orc_poisson_square(n, tol, _ptr(F), _ptr(X))
    return X


def rect_scales(width: float, height: float):
    """(kx, ky) = ((2/width)^2, (2/height)^2): the factors the affine map of
    [x0, x0 + width] x [y0, y0 + height] onto [-1, 1]^2 puts on u_xx and u_yy."""
    return (2.0 / width) ** 2, (2.0 / height) ** 2


def poisson_rectangle(F, width: float, height: float, tol: float = 1e-13, variant: str = "double",
                      tight: bool = False):
    """Poisson on a width x height rectangle, homogeneous Dirichlet data:
    kx M X D^T + ky D X M^T = F, F and X in the mapped C~ basis (X_ij pairs C~_i(y)
    with C~_j(x)).  Returns (X, J)."""
    F = _f64(F)
    n = F.shape[0]
    X = np.zeros_like(F)
    kx, ky = rect_scales(width, height)
    J = _lib(variant).orc_poisson_rectangle(n, kx, ky, tol, 1 if tight else 0, _ptr(F), _ptr(X))
    return X, int(J)


def tight_interval(n: int):
    """(lo, hi) with sigma(A~) in [-hi, -lo]: Sturm-count bisection on the even and odd
    tridiagonals of A~, padded (lo = |lambda_max|/2, hi = min(1, 1.01 |lambda_min|))."""
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _lib().orc_tight_interval(int(n), ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def poisson_square_partial(F, tol: float, jmax: int) -> np.ndarray:
    """The pipeline of poisson_square stopped after at most jmax ADI iterations."""
    F = _f64(F)
    n = F.shape[0]
    X = np.zeros_like(F)
    _lib().orc_poisson_square_partial(n, tol, int(jmax), _ptr(F), _ptr(X))
    return X


def poisson_cube(F, tol: float = 1e-13, tol_mid: float = 1e-15, tol_in: float = 1e-15, variant: str = "double"):
    """Solve (5.2) on the cube by the nested ADI of Sec. 5.  Returns (X, J_outer, inner
    iterations over full tensors)."""
    F = _f64(F)
    n = F.shape[0]
    assert F.shape == (n, n, n)
    X = np.zeros_like(F)
    J = ctypes.c_int()
    inner = _lib(variant).orc_poisson_cube(n, tol, tol_mid, tol_in, _ptr(F), _ptr(X), ctypes.byref(J))
    return X, J.value, int(inner)


def square_iterations(n: int, tol: float) -> int:
    a, b, c, d = square_interval(n)
    return adi_iterations(a, b, c, d, tol)


def num_threads() -> int:
    return int(_lib().orc_num_threads())


def set_num_threads(t: int) -> None:
    for v in list(_LIBS):
        _LIBS[v].orc_set_num_threads(int(t))
    _lib().orc_set_num_threads(int(t))


def real_bytes(variant: str = "double") -> int:
    return int(_lib(variant).orc_real_bytes())


if __name__ == "__main__":  # pragma: no cover
    build()
    print("oracle built in", _BUILD, file=sys.stderr)


# --------------------------------------------------------------------------
# Sec. 3.4 / Table 3.1 steps 1 and 4: Legendre coefficients in and out
# --------------------------------------------------------------------------
def legendre_to_ctilde(G) -> np.ndarray:
    """F = B G B^T: C~ coefficients of sum G_ab P_a(y) P_b(x) (n x n)."""
    G = _f64(G)
    n = G.shape[0]
    F = np.zeros_like(G)
    _lib().orc_legendre_to_ctilde(n, _ptr(G), _ptr(F))
    return F


def solution_to_legendre(X) -> np.ndarray:
    """Legendre coefficients ((n+2) x (n+2)) of u = (1-x^2)(1-y^2) sum X_ij C~_i(y) C~_j(x)."""
    X = _f64(X)
    n = X.shape[0]
    U = np.zeros((n + 2, n + 2))
    _lib().orc_solution_to_legendre(n, _ptr(X), _ptr(U))
    return U


def legendre_to_ctilde_adjoint(Fbar) -> np.ndarray:
    """Gbar = B^T Fbar B, the transpose of ``legendre_to_ctilde`` (n x n)."""
    Fbar = _f64(Fbar)
    n = Fbar.shape[0]
    Gbar = np.zeros_like(Fbar)
    _lib().orc_legendre_to_ctilde_adjoint(n, _ptr(Fbar), _ptr(Gbar))
    return Gbar


def solution_to_legendre_adjoint(Ubar) -> np.ndarray:
    """Xbar (n x n) = M^T B^{-T} Ubar B^{-1} M, the transpose of ``solution_to_legendre``
    (Ubar is (n+2) x (n+2))."""
    Ubar = _f64(Ubar)
    n = Ubar.shape[0] - 2
    Xbar = np.zeros((n, n))
    _lib().orc_solution_to_legendre_adjoint(n, _ptr(Ubar), _ptr(Xbar))
    return Xbar
