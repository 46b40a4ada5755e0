"""Oracle for the cylinder's Fourier modes |k| >= 2 (Sec. 4.1, Case 1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): imported by the tests, the
smoke check and the CPU legs of the benchmark, never by the GPU library.

After the doubling-up of Sec. 4.1 each Fourier mode k of the solution is written
u_k(r, z) = r^2 (1 - r^2)(1 - z^2) w_k(r, z) with
    w_k = sum_{i,j < n} Y[i, j] C~_i(r) C~_j(z),
and substituting into u_rr + u_r / r - k^2 u / r^2 + u_zz = f_k gives
    [L1 w - k^2 (1 - r^2) w] (1 - z^2) + r^2 (1 - r^2) L2 w = f_k,
    L1 = r^2 (1 - r^2) d^2/dr^2 + (5 - 9 r^2) r d/dr + 4 (1 - 4 r^2),
    L2 = (1 - z^2) d^2/dz^2 - 4 z d/dz - 2   (L2 C~_j = D_jj C~_j, D_jj = -(j+1)(j+2)).
With F the C~ x C~ coefficients of f_k the coefficients satisfy
    P Y M^T + Q Y D = F,   P = L1 - k^2 M,  Q = matrix of r^2 (1 - r^2),  M of (1 - r^2),
i.e. A Y - Y B = P^{-1} F D^{-1} with A = P^{-1} Q and B = -M D^{-1}.  (The factor
r^2 of Q is dropped in the printed A; the equation before the rearrangement keeps it,
and so does this module.)  Every matrix here is the n x n block of its operator, built
from the definition: C~_a against the operator applied to C~_i, integrated by
Gauss-Jacobi(1, 1) quadrature, with derivatives of C^(3/2) from
d/dx C^(l)_m = 2 l C^(l+1)_{m-1} (DLMF 18.9.19).
"""
from __future__ import annotations

import numpy as np
from scipy.special import eval_gegenbauer, roots_jacobi

from . import adi_iterations, adi_shifts


def _ct(j: int, x: np.ndarray, d: int = 0) -> np.ndarray:
    """d-th derivative of C~_j = s_j C_j^(3/2) at x."""
    s = np.sqrt((j + 1.5) / ((j + 1.0) * (j + 2.0)))
    if d == 0:
        return s * eval_gegenbauer(j, 1.5, x)
    if d == 1:
        return s * 3.0 * eval_gegenbauer(j - 1, 2.5, x) if j >= 1 else 0.0 * x
    return s * 15.0 * eval_gegenbauer(j - 2, 3.5, x) if j >= 2 else 0.0 * x


def _operator(n: int, apply) -> np.ndarray:
    """T[a, i] = int C~_a (apply C~_i) (1 - x^2) dx, a, i < n (the n x n block)."""
    x, w = roots_jacobi(n + 8, 1.0, 1.0)
    Bm = np.stack([_ct(a, x) for a in range(n)])
    V = np.stack([apply(i, x) for i in range(n)])
    return (Bm * w) @ V.T


def mode_operators(n: int, k: int):
    """(P, Q, M, D): P = L1 - k^2 M, Q = r^2 (1 - r^2), M = (1 - r^2), D = diag(-(j+1)(j+2))."""
    M = _operator(n, lambda i, x: (1 - x * x) * _ct(i, x))
    Q = _operator(n, lambda i, x: x * x * (1 - x * x) * _ct(i, x))
    L1 = _operator(n, lambda i, x: x * x * (1 - x * x) * _ct(i, x, 2) + (5 - 9 * x * x) * x * _ct(i, x, 1)
                   + 4 * (1 - 4 * x * x) * _ct(i, x))
    D = np.diag([-(j + 1.0) * (j + 2.0) for j in range(n)])
    return L1 - k * k * M, Q, M, D


def l1_matrix(n: int) -> np.ndarray:
    """L1 alone (the matrix of the r-operator of Case 1)."""
    P, _, M, _ = mode_operators(n, 0)
    return P


def mode_solve_dense(F, k: int) -> np.ndarray:
    """Exact discrete solution of P Y M^T + Q Y D = F by a Kronecker solve (small n)."""
    F = np.asarray(F, dtype=np.float64)
    n = F.shape[0]
    P, Q, M, D = mode_operators(n, k)
    K = np.kron(P, M) + np.kron(Q, D)
    return np.linalg.solve(K, F.reshape(-1)).reshape(n, n)


def mode_intervals(n: int, k: int, pad: float = 0.02):
    """Intervals [a, b] containing sigma(A) (negative) and [c, d] containing sigma(B)
    (positive), from the dense eigenvalues, widened by `pad` on the outside."""
    P, Q, M, D = mode_operators(n, k)
    ea = np.linalg.eigvals(np.linalg.solve(P, Q))
    eb = np.linalg.eigvals(-M @ np.linalg.inv(D))
    assert np.abs(ea.imag).max() <= 1e-10 * np.abs(ea).max() and np.abs(eb.imag).max() <= 1e-12
    a, b = ea.real.min() * (1 + pad), ea.real.max() * (1 - pad)
    c, d = eb.real.min() * (1 - pad), eb.real.max() * (1 + pad)
    assert a < b < 0 < c < d
    return a, b, c, d


def mode_adi(F, k: int, tol: float = 1e-13, intervals=None):
    """The ADI iteration of Algorithm 2 on A Y - Y B = C, C = P^{-1} F D^{-1} (the
    first half-step in the form X_{j+1/2}(B - p_j) = (A - p_j) X_j - C), shifts (2.4)
    from the intervals of ``mode_intervals`` and J from (2.9).  Dense algebra per step;
    returns (Y, J)."""
    F = np.asarray(F, dtype=np.float64)
    n = F.shape[0]
    P, Q, M, D = mode_operators(n, k)
    a, b, c, d = intervals if intervals is not None else mode_intervals(n, k)
    J = adi_iterations(a, b, c, d, tol)
    p, q = adi_shifts(a, b, c, d, tol, J)
    A = np.linalg.solve(P, Q)
    B = -M @ np.linalg.inv(D)
    C = np.linalg.solve(P, F) @ np.linalg.inv(D)
    I = np.eye(n)
    X = np.zeros((n, n))
    for j in range(J):
        Xh = np.linalg.solve((B - p[j] * I).T, ((A - p[j] * I) @ X - C).T).T
        X = np.linalg.solve(A - q[j] * I, Xh @ (B - q[j] * I) + C)
    return X, J
