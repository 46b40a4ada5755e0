"""Normalised ultraspherical basis C~^(3/2) and Gauss quadrature (test infrastructure).

The basis is defined in the footnote of Sec. 3.1:
    C~_j(x) = sqrt((j + 3/2) / ((j+1)(j+2))) C_j^(3/2)(x),
orthonormal on [-1, 1] for the weight (1 - x^2).  Coefficients of a function g
in this basis are  g_j = int g(x) C~_j(x) (1 - x^2) dx, evaluated here with
Gauss-Jacobi(1, 1) quadrature (exact for polynomial integrands of degree
< 2N).  Used to build manufactured right-hand sides and exact solutions from
the ansatz (3.2), and to pin the multiplication matrix M of (3.7).
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import polynomial as P
from scipy.special import eval_gegenbauer, roots_jacobi


def ctilde(j: int, x: np.ndarray) -> np.ndarray:
    """C~_j^(3/2)(x) (footnote of Sec. 3.1)."""
    return np.sqrt((j + 1.5) / ((j + 1.0) * (j + 2.0))) * eval_gegenbauer(j, 1.5, x)


def basis_matrix(n: int, x: np.ndarray) -> np.ndarray:
    """B[j, a] = C~_j(x_a) for j < n."""
    return np.stack([ctilde(j, x) for j in range(n)])


def gauss_jacobi(N: int):
    """Nodes and weights for int f(x) (1 - x^2) dx."""
    x, w = roots_jacobi(N, 1.0, 1.0)
    return x, w


def project_1d(values_fn, n: int, N: int) -> np.ndarray:
    """Coefficients g_j = int g C~_j (1-x^2) dx for j < n."""
    x, w = gauss_jacobi(N)
    return basis_matrix(n, x) @ (w * values_fn(x))


def project_2d(f, n: int, N: int) -> np.ndarray:
    """F[i, j] = int int f(x, y) C~_i(y) C~_j(x) (1-x^2)(1-y^2) dx dy.

    Row index i pairs with y and column index j with x, as in (3.2)."""
    x, w = gauss_jacobi(N)
    Bm = basis_matrix(n, x)                    # [j, a]
    Xg, Yg = np.meshgrid(x, x, indexing="xy")  # Xg[a_y, a_x] = x[a_x], Yg[a_y, a_x] = x[a_y]
    vals = f(Xg, Yg)                           # vals[a_y, a_x]
    return (Bm * w) @ vals @ (Bm * w).T


# --------------------------------------------------------------------------
# Polynomials in two variables: coefficient arrays c[a, b] of x^a y^b.
# --------------------------------------------------------------------------
def poly_times_bubble(c: np.ndarray) -> np.ndarray:
    """(1 - x^2)(1 - y^2) p(x, y) for p given by c[a, b] (x^a y^b)."""
    one_minus_sq = np.array([1.0, 0.0, -1.0])
    out = np.zeros((c.shape[0] + 2, c.shape[1] + 2))
    for a in range(c.shape[0]):
        for b in range(c.shape[1]):
            if c[a, b] != 0.0:
                out[a:a + 3, b:b + 3] += c[a, b] * np.outer(one_minus_sq, one_minus_sq)
    return out


def laplacian(c: np.ndarray) -> np.ndarray:
    """u_xx + u_yy for u given by c[a, b] (x^a y^b)."""
    uxx = P.polyder(c, 2, axis=0)
    uyy = P.polyder(c, 2, axis=1)
    out = np.zeros(c.shape)
    out[: uxx.shape[0], : uxx.shape[1]] += uxx
    out[: uyy.shape[0], : uyy.shape[1]] += uyy
    return out


def poly_eval(c: np.ndarray, X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    return P.polyval2d(X, Y, c)


def manufactured_rectangle(pc: np.ndarray, n: int, kx: float, ky: float):
    """As manufactured_square on the mapped rectangle: u = (1-s^2)(1-t^2) p(s,t) in the
    coordinates s (x) and t (y) of [-1,1]^2, and f = kx u_ss + ky u_tt, the Laplacian
    of u on a rectangle whose side lengths are 2/sqrt(kx) and 2/sqrt(ky)."""
    u = poly_times_bubble(pc)
    uxx = P.polyder(u, 2, axis=0)
    uyy = P.polyder(u, 2, axis=1)
    f = np.zeros(u.shape)
    f[: uxx.shape[0], : uxx.shape[1]] += kx * uxx
    f[: uyy.shape[0], : uyy.shape[1]] += ky * uyy
    deg = u.shape[0] + u.shape[1]
    N = n + deg + 4
    F = project_2d(lambda X, Y: poly_eval(f, X, Y), n, N)
    Xe = project_2d(lambda X, Y: poly_eval(pc, X, Y), n, N)
    return F, Xe


def manufactured_square(pc: np.ndarray, n: int):
    """Manufactured pair for eq. (3.1): u = (1-x^2)(1-y^2) p(x,y).

    Returns (F, X_exact): F the C~ coefficients of f = Laplacian(u) and
    X_exact the C~ coefficients of p, so that u has the expansion (3.2) with
    coefficients X_exact.  Exact (up to rounding) when deg p + 2 < n."""
    u = poly_times_bubble(pc)
    f = laplacian(u)
    deg = u.shape[0] + u.shape[1]
    N = n + deg + 4
    F = project_2d(lambda X, Y: poly_eval(f, X, Y), n, N)
    Xe = project_2d(lambda X, Y: poly_eval(pc, X, Y), n, N)
    return F, Xe


def monomial_coeffs(values: np.ndarray, deg: int) -> np.ndarray:
    """Arrange coefficients of the monomials x^a y^b with a + b <= deg, ordered by
    total degree t = 0..deg and, within a degree, by a descending, into c[a, b]."""
    c = np.zeros((deg + 1, deg + 1))
    k = 0
    for t in range(deg + 1):
        for a in range(t, -1, -1):
            c[a, t - a] = values[k]
            k += 1
    assert k == len(values)
    return c


# --------------------------------------------------------------------------
# The cube: u = (1-x^2)(1-y^2)(1-z^2) p(x, y, z), coefficients c[a, b, g] of x^a y^b z^g.
# Tensor index order (x, y, z): X[i, j, k] pairs C~_i(x) C~_j(y) C~_k(z).
# --------------------------------------------------------------------------
def project_3d(f, n: int, N: int) -> np.ndarray:
    """F[i, j, k] = int f(x,y,z) C~_i(x) C~_j(y) C~_k(z) (1-x^2)(1-y^2)(1-z^2)."""
    x, w = gauss_jacobi(N)
    Bm = basis_matrix(n, x) * w                      # [j, a]
    Xg, Yg, Zg = np.meshgrid(x, x, x, indexing="ij")
    vals = f(Xg, Yg, Zg)
    return np.einsum("ia,jb,kc,abc->ijk", Bm, Bm, Bm, vals)


def _poly3_eval(c, X, Y, Z):
    out = np.zeros_like(X)
    for a in range(c.shape[0]):
        for b in range(c.shape[1]):
            for g in range(c.shape[2]):
                if c[a, b, g] != 0.0:
                    out += c[a, b, g] * X**a * Y**b * Z**g
    return out


def _poly3_bubble(c):
    bub = np.array([1.0, 0.0, -1.0])
    out = np.zeros((c.shape[0] + 2, c.shape[1] + 2, c.shape[2] + 2))
    for a in range(c.shape[0]):
        for b in range(c.shape[1]):
            for g in range(c.shape[2]):
                if c[a, b, g] != 0.0:
                    out[a:a + 3, b:b + 3, g:g + 3] += c[a, b, g] * np.einsum("a,b,c->abc", bub, bub, bub)
    return out


def _poly3_laplacian(c):
    out = np.zeros(c.shape)
    for ax in range(3):
        dd = P.polyder(c, 2, axis=ax)
        sl = tuple(slice(0, s) for s in dd.shape)
        out[sl] += dd
    return out


def manufactured_cube(pc: np.ndarray, n: int):
    """(F, X_exact) for u = (1-x^2)(1-y^2)(1-z^2) p with p given by pc[a, b, g]."""
    u = _poly3_bubble(pc)
    f = _poly3_laplacian(u)
    N = n + sum(u.shape) + 2
    F = project_3d(lambda X, Y, Z: _poly3_eval(f, X, Y, Z), n, N)
    Xe = project_3d(lambda X, Y, Z: _poly3_eval(pc, X, Y, Z), n, N)
    return F, Xe
