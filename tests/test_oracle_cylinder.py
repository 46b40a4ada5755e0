"""Pins of the cylinder oracle (Sec. 4.1, Case 1) against things other than itself:
the change of variables checked symbolically from the cylindrical Laplacian (sympy),
manufactured polynomial solutions whose right-hand sides come from that Laplacian
(never from the oracle's matrices), the band structure and operator identity of L1
(including the constant the printed formula gets wrong), and the ADI against the
Kronecker solve."""
import numpy as np
import pytest
import sympy as sp
from scipy.special import roots_jacobi

from oracle import basis
from oracle import cylinder as cyl

r, z, kk = sp.symbols("r z k")


def _omega(deg, par, seed):
    """A random polynomial w(r, z) of degree <= deg in each variable, of parity `par` in r."""
    rng = np.random.default_rng(seed)
    terms = 0
    for a in range(par, deg + 1, 2):
        for b in range(deg + 1):
            terms += sp.Rational(int(rng.integers(-9, 10)), 7) * r ** a * z ** b
    return terms


def test_change_of_variables_symbolic():
    """u = r^2 (1-r^2)(1-z^2) w: u_rr + u_r/r - k^2 u/r^2 + u_zz equals
    [L1 w - k^2 (1-r^2) w](1-z^2) + r^2(1-r^2) L2 w for every w."""
    w = sp.Function("w")(r, z)
    u = r ** 2 * (1 - r ** 2) * (1 - z ** 2) * w
    lap = sp.diff(u, r, 2) + sp.diff(u, r) / r - kk ** 2 * u / r ** 2 + sp.diff(u, z, 2)
    L1w = r ** 2 * (1 - r ** 2) * sp.diff(w, r, 2) + (5 - 9 * r ** 2) * r * sp.diff(w, r) + 4 * (1 - 4 * r ** 2) * w
    L2w = (1 - z ** 2) * sp.diff(w, z, 2) - 4 * z * sp.diff(w, z) - 2 * w
    rhs = (L1w - kk ** 2 * (1 - r ** 2) * w) * (1 - z ** 2) + r ** 2 * (1 - r ** 2) * L2w
    assert sp.simplify(sp.expand(lap - rhs)) == 0


def test_l1_bands_and_operator_identity():
    """L1 has bands 0 and +-2 only (tridiagonal in each parity) and equals
    M_{r^2} D + 5 M_r M D_1 + 14 M - 10 I; the printed -6 I is off by 4 I."""
    n = 20
    L1 = cyl.l1_matrix(n)
    for off in range(-n + 1, n):
        if off not in (-2, 0, 2):
            assert np.abs(np.diag(L1, off)).max() <= 1e-10, off
    _, Q, M, D = cyl.mode_operators(n, 0)
    X1 = cyl._operator(n, lambda i, x: x * (1 - x * x) * cyl._ct(i, x, 1))  # r (1 - r^2) d/dr
    I = np.eye(n)
    built = (I - M) @ D + 5 * X1 + 14 * M - 10 * I
    # (I - M) D is exact in the n x n block except where M's band +2 leaves it
    assert np.abs(L1 - built)[: n - 2, : n - 2].max() <= 1e-10
    assert np.allclose(((I - M) @ D + 5 * X1 + 14 * M - 6 * I - L1)[: n - 2, : n - 2], 4 * I[: n - 2, : n - 2],
                       atol=1e-9)
    for off in range(-n + 1, n):
        if abs(off) > 4 or off % 2:
            assert np.abs(np.diag(Q, off)).max() <= 1e-12, off


def _project2(fn, n, N):
    """C~ x C~ coefficients of fn(r, z) (row index = degree in r)."""
    x, w = roots_jacobi(N, 1.0, 1.0)
    Bm = basis.basis_matrix(n, x)
    R, Z = np.meshgrid(x, x, indexing="ij")
    return (Bm * w) @ fn(R, Z) @ (Bm * w).T


@pytest.mark.parametrize("k,deg", [(2, 6), (3, 7), (6, 9), (11, 5)])
def test_manufactured_solution(k, deg):
    """w polynomial of parity k in r: F from the cylindrical Laplacian of
    u = r^2(1-r^2)(1-z^2) w (symbolic, then projected), Y must be w's coefficients."""
    n = deg + 3
    w = _omega(deg, k % 2, 10 + k)
    u = r ** 2 * (1 - r ** 2) * (1 - z ** 2) * w
    f = sp.expand(sp.diff(u, r, 2) + sp.diff(u, r) / r - k ** 2 * u / r ** 2 + sp.diff(u, z, 2))
    f_num = sp.lambdify((r, z), f, "numpy")
    w_num = sp.lambdify((r, z), w, "numpy")
    F = _project2(lambda R, Z: f_num(R, Z) + 0 * R, n, n + 12)
    Y_true = _project2(lambda R, Z: w_num(R, Z) + 0 * R, n, n + 12)
    Y = cyl.mode_solve_dense(F, k)
    assert np.abs(Y - Y_true).max() <= 1e-11 * np.abs(Y_true).max()
    Ya, J = cyl.mode_adi(F, k, 1e-14)
    assert np.abs(Ya - Y_true).max() <= 1e-10 * np.abs(Y_true).max()


@pytest.mark.parametrize("n,k", [(16, 2), (24, 3), (24, 9), (40, 20)])
def test_adi_against_kronecker(n, k):
    """The ADI with the Zolotarev shifts of the dense eigenvalue intervals reaches the
    Kronecker solution; A is only near-normal (eigenvector condition kappa), so the
    bar is tol x kappa x 10."""
    F = np.random.default_rng(n + k).standard_normal((n, n)) / np.add.outer(np.arange(n) + 1.0,
                                                                              np.arange(n) + 1.0) ** 2
    tol = 1e-12
    P, Q, M, D = cyl.mode_operators(n, k)
    kappa = np.linalg.cond(np.linalg.eig(np.linalg.solve(P, Q))[1])
    Y, J = cyl.mode_adi(F, k, tol)
    Ye = cyl.mode_solve_dense(F, k)
    assert np.abs(Y - Ye).max() <= 10 * tol * kappa * np.abs(Ye).max(), (J, kappa)


def test_intervals_disjoint_and_contain_spectra():
    for n, k in [(16, 2), (32, 5), (48, 24)]:
        a, b, c, d = cyl.mode_intervals(n, k)
        P, Q, M, D = cyl.mode_operators(n, k)
        ea = np.linalg.eigvals(np.linalg.solve(P, Q)).real
        assert a <= ea.min() and ea.max() <= b < 0 < c
