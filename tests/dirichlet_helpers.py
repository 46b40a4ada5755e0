"""Helpers of the Dirichlet tests that route around the oracle: traces of a
Legendre expansion by P_k(+-1) = (+-1)^k, and the Laplacian of an expansion by two
routes that share nothing with the oracle's differentiation (power basis; the
Legendre equation at Gauss nodes with quadrature projection)."""
import numpy as np
from numpy.polynomial import legendre as npleg
from numpy.polynomial import polynomial as nppoly


def traces(U):
    """Traces [g_W, g_E, g_S, g_N] of u = sum U[i, j] P_i(y) P_j(x) (P_k(+-1) = (+-1)^k)."""
    m = U.shape[0]
    alt = (-1.0) ** np.arange(m)
    one = np.ones(m)
    return np.stack([U @ alt, U @ one, alt @ U, one @ U])


def fixed_length(fn, v):
    out = np.zeros(len(v))
    r = fn(v)
    out[: len(r)] = r
    return out


def along_both(fn, C):
    C = np.apply_along_axis(lambda v: fixed_length(fn, v), 0, C)
    return np.apply_along_axis(lambda v: fixed_length(fn, v), 1, C)


def laplacian_power_route(U, kx, ky):
    """Legendre coefficients of kx u_xx + ky u_yy computed through the power basis
    (leg2poly, polyder, poly2leg): an independent route to the derivative."""
    P = along_both(npleg.leg2poly, U)
    m = U.shape[0]
    Pyy = np.zeros_like(P)
    Pxx = np.zeros_like(P)
    d = nppoly.polyder(P, 2, axis=0)
    Pyy[: d.shape[0], :] = d
    d = nppoly.polyder(P, 2, axis=1)
    Pxx[:, : d.shape[1]] = d
    return along_both(npleg.poly2leg, ky * Pyy + kx * Pxx)


def laplacian_by_quadrature(U, kx, ky):
    """Legendre coefficients of kx u_xx + ky u_yy by Gauss-Legendre projection of its
    values, with P_j'' at the (interior) nodes from the Legendre equation,
    (1-x^2) P'' = 2x P' - j(j+1) P and (1-x^2) P' = j (P_{j-1} - x P_j): a route that
    uses no differentiation of coefficient series and stays accurate at high degree."""
    m = U.shape[0]
    x, w = npleg.leggauss(m + 4)
    V = npleg.legvander(x, m)                       # P_0 .. P_m at the nodes
    j = np.arange(m)
    s = (1 - x * x)[:, None]
    Pm1 = np.hstack([np.zeros((len(x), 1)), V[:, : m - 1]])
    dV = j * (Pm1 - x[:, None] * V[:, :m]) / s
    d2V = (2 * x[:, None] * dV - j * (j + 1) * V[:, :m]) / s
    Vm = V[:, :m]
    Fv = kx * Vm @ U @ d2V.T + ky * d2V @ U @ Vm.T  # values at (y_a, x_b)
    Pw = Vm * w[:, None] * (2 * j + 1) / 2.0
    return Pw.T @ Fv @ Pw
