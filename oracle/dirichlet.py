"""Oracle for nonhomogeneous Dirichlet data (Sec. 6.1) on the square or a rectangle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): imported by the tests, the
smoke check and the CPU legs of the benchmark, never by the GPU library.

Sec. 6.1 moves the boundary data into the right-hand side in four steps:
  1. coefficients X_bc of some function u_bc that takes the Dirichlet data,
  2. its Laplacian,
  3. the homogeneous solve of  lap u_rhs = f - lap u_bc,
  4. X = X_rhs + X_bc.
The paper leaves the choice of u_bc open.  Here it is the transfinite (Coons)
interpolant of the four side traces,
  u_bc = P_x + P_y - P_x P_y,
  P_x  = (1-x)/2 g_W(y) + (1+x)/2 g_E(y),   P_y = (1-y)/2 g_S(x) + (1+y)/2 g_N(x),
  P_x P_y = the bilinear interpolant of the four corner values,
each corner value the mean of the two traces meeting there (with data that agree at
the corners u_bc takes every trace exactly).  Everything is in Legendre
coefficients of the mapped variables x, y in [-1, 1]: f = sum G[a, b] P_a(y) P_b(x)
(n x n), traces g_W = u(-1, y), g_E = u(1, y), g_S = u(x, -1), g_N = u(x, 1) with n+2
coefficients each (rows of ``bc`` in that order), and the solution
u = sum U[i, j] P_i(y) P_j(x) with (n+2) x (n+2) coefficients, the size Table 3.1's
step 4 returns.  On a width x height rectangle the Laplacian in the mapped variables
is kx d^2/dx^2 + ky d^2/dy^2 with (kx, ky) = ((2/width)^2, (2/height)^2).

The Laplacian of u_bc is taken with numpy's Legendre differentiation and cut to the
n x n block the input map takes (exact for n >= 2: the second derivative along one
variable lowers its degree by two, and the other variable keeps degree <= 1).
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npleg

from . import (legendre_to_ctilde, legendre_to_ctilde_adjoint, poisson_rectangle, poisson_square,
               rect_scales, solution_to_legendre, solution_to_legendre_adjoint)

SIDES = ("W", "E", "S", "N")


def _corners(bc):
    """Corner values c[(sx, sy)] = mean of the two traces meeting at (x, y) = (sx, sy)."""
    gW, gE, gS, gN = (np.asarray(b, dtype=np.float64) for b in bc)
    val = lambda g, s: float(npleg.legval(float(s), g))
    return {(-1, -1): 0.5 * (val(gW, -1) + val(gS, -1)),
            (-1, 1): 0.5 * (val(gW, 1) + val(gN, -1)),
            (1, -1): 0.5 * (val(gE, -1) + val(gS, 1)),
            (1, 1): 0.5 * (val(gE, 1) + val(gN, 1))}


def lift(bc) -> np.ndarray:
    """Step 1: Legendre coefficients ((n+2) x (n+2); row = degree in y) of the Coons
    interpolant u_bc of the traces bc = [g_W, g_E, g_S, g_N] (each n+2 long)."""
    bc = np.asarray(bc, dtype=np.float64)
    m = bc.shape[1]
    gW, gE, gS, gN = bc
    # linear factors in Legendre form: (1 - t)/2 = P_0/2 - P_1/2, (1 + t)/2 = P_0/2 + P_1/2
    lo = np.zeros(m)
    hi = np.zeros(m)
    lo[0], lo[1] = 0.5, -0.5
    hi[0], hi[1] = 0.5, 0.5
    Xbc = np.outer(gW, lo) + np.outer(gE, hi)        # P_x: traces in y times linear factors in x
    Xbc += np.outer(lo, gS) + np.outer(hi, gN)       # P_y
    c = _corners(bc)
    fac = {-1: lo, 1: hi}
    for (sx, sy), v in c.items():                    # - P_x P_y
        Xbc -= v * np.outer(fac[sy], fac[sx])
    return Xbc


def lift_laplacian(bc, kx: float = 1.0, ky: float = 1.0) -> np.ndarray:
    """Step 2: Legendre coefficients (n x n) of kx u_bc,xx + ky u_bc,yy."""
    Xbc = lift(bc)
    n = Xbc.shape[0] - 2
    Lyy = npleg.legder(Xbc, 2, axis=0)               # (n) x (n+2)
    Lxx = npleg.legder(Xbc, 2, axis=1)               # (n+2) x (n)
    return ky * Lyy[:n, :n] + kx * Lxx[:n, :n]


def _solve(F, width: float, height: float, tol: float):
    if width == 2.0 and height == 2.0:
        return poisson_square(F, tol)
    return poisson_rectangle(F, width, height, tol)[0]


def poisson_dirichlet(G, bc, width: float = 2.0, height: float = 2.0, tol: float = 1e-13) -> np.ndarray:
    """Steps 1-4 of Sec. 6.1 with Table 3.1 around the homogeneous solve: returns U,
    the (n+2) x (n+2) Legendre coefficients of u."""
    G = np.asarray(G, dtype=np.float64)
    kx, ky = rect_scales(width, height)
    Gm = G - lift_laplacian(bc, kx, ky)              # f - lap u_bc
    X = _solve(legendre_to_ctilde(Gm), width, height, tol)
    return solution_to_legendre(X) + lift(bc)


def _lift_matrix_T(Ubar) -> np.ndarray:
    """Transpose of ``lift`` applied to Ubar ((n+2) x (n+2)): the gradient in bc."""
    Ubar = np.asarray(Ubar, dtype=np.float64)
    m = Ubar.shape[0]
    lo = np.zeros(m)
    hi = np.zeros(m)
    lo[0], lo[1] = 0.5, -0.5
    hi[0], hi[1] = 0.5, 0.5
    g = np.zeros((4, m))
    g[0] = Ubar @ lo
    g[1] = Ubar @ hi
    g[2] = lo @ Ubar
    g[3] = hi @ Ubar
    # corners: d/dc(sx, sy) of -sum Ubar * c * outer(fac[sy], fac[sx]); c = mean of trace values
    fac = {-1: lo, 1: hi}
    ev = lambda s: np.array([float(s) ** k for k in range(m)])   # d trace(s) / d coefficients
    side_of = {(-1, -1): ((0, -1), (2, -1)), (-1, 1): ((0, 1), (3, -1)),
               (1, -1): ((1, -1), (2, 1)), (1, 1): ((1, 1), (3, 1))}
    for (sx, sy), pairs in side_of.items():
        cbar = -float(fac[sy] @ Ubar @ fac[sx])
        for side, s in pairs:
            g[side] += 0.5 * cbar * ev(s)
    return g


def _d2_matrix(m: int) -> np.ndarray:
    """Second derivative of a Legendre series with m coefficients, as an m x m matrix
    (columns: numpy's derivative of each unit series, padded with zeros)."""
    D = np.zeros((m, m))
    D[: max(m - 2, 0), :] = npleg.legder(np.eye(m), 2, axis=0) if m > 2 else 0.0
    return D


def poisson_dirichlet_adjoint(Ubar, width: float = 2.0, height: float = 2.0, tol: float = 1e-13):
    """Gradients (dL/dG, dL/dbc) of a loss L(U) from dL/dU: the transpose of the linear
    map (G, bc) -> U of ``poisson_dirichlet``, composed step by step in reverse."""
    Ubar = np.asarray(Ubar, dtype=np.float64)
    Xbar = solution_to_legendre_adjoint(Ubar)
    Fbar = _solve(Xbar, width, height, tol)          # the solve map is self-adjoint
    Gbar = legendre_to_ctilde_adjoint(Fbar)
    return Gbar, traces_adjoint(Ubar, Gbar, width, height)


def traces_adjoint(Ubar, Gbar, width: float = 2.0, height: float = 2.0) -> np.ndarray:
    """The gradient in the traces given dL/dU and dL/dG: U depends on bc through the
    lift (directly) and through -lift_laplacian in the right-hand side;
    lap = ky D2 Xbc + kx Xbc D2^T cut to n x n, whose transpose sends Gbar to
    ky D2^T Gp + kx Gp D2 (Gp = Gbar padded to m x m)."""
    Ubar = np.asarray(Ubar, dtype=np.float64)
    m = Ubar.shape[0]
    n = m - 2
    kx, ky = rect_scales(width, height)
    D2 = _d2_matrix(m)
    Gp = np.zeros((m, m))
    Gp[:n, :n] = Gbar
    Xbc_bar = Ubar - (ky * D2.T @ Gp + kx * Gp @ D2)
    return _lift_matrix_T(Xbc_bar)
