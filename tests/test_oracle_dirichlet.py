"""Pins of the oracle for nonhomogeneous Dirichlet data (Sec. 6.1) and of the
transposed Legendre maps, each against something other than the oracle itself:
evaluation of the lifted function on the boundary, power-basis differentiation,
manufactured polynomial solutions, convergence to a smooth non-polynomial solution
evaluated pointwise, and the defining identity of a transpose (<A x, y> = <x, A^T y>)
checked with the forward maps, including an exhaustive Jacobian at n = 3."""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

import oracle
from oracle import dirichlet as odir
from dirichlet_helpers import laplacian_by_quadrature, laplacian_power_route, traces

RECTS = [(2.0, 2.0), (3.0, 0.75), (0.5, 4.0)]


def _random_compatible_bc(n, seed):
    rng = np.random.default_rng(seed)
    m = n + 2
    U = rng.standard_normal((m, m)) / np.add.outer(np.arange(m) + 1.0, np.arange(m) + 1.0) ** 2
    return traces(U)


@pytest.mark.parametrize("n", [1, 2, 5, 16])
def test_lift_takes_the_traces(n):
    bc = _random_compatible_bc(n, 3)
    Xbc = odir.lift(bc)
    t = np.linspace(-1, 1, 41)
    one = np.ones_like(t)
    for side, (x, y) in enumerate([(-one, t), (one, t), (t, -one), (t, one)]):
        got = npleg.legval2d(y, x, Xbc)
        want = npleg.legval(t, bc[side])
        assert np.allclose(got, want, atol=1e-13 * max(1.0, np.abs(want).max())), side


def test_lift_uses_corner_means_for_incompatible_data():
    """With traces that disagree at a corner the lift takes the mean there."""
    n = 4
    bc = np.zeros((4, n + 2))
    bc[0, 0] = 1.0   # g_W = 1, all other traces 0: corners (-1, +-1) disagree
    Xbc = odir.lift(bc)
    for x, y in [(-1, -1), (-1, 1)]:
        assert abs(npleg.legval2d(y, x, Xbc) - 0.5) < 1e-15
    assert abs(npleg.legval2d(0.0, -1.0, Xbc) - 0.5) < 1e-15   # mid-side: mean of the corner values


@pytest.mark.parametrize("w,h", RECTS)
def test_lift_laplacian_against_power_basis(w, h):
    n = 14
    kx, ky = oracle.rect_scales(w, h)
    bc = _random_compatible_bc(n, 5)
    L = odir.lift_laplacian(bc, kx, ky)
    want = laplacian_power_route(odir.lift(bc), kx, ky)
    assert np.abs(want[n:, :]).max() < 1e-12 and np.abs(want[:, n:]).max() < 1e-12
    assert np.allclose(L, want[:n, :n], rtol=0, atol=1e-11 * np.abs(want).max())
    want2 = laplacian_by_quadrature(odir.lift(bc), kx, ky)
    assert np.allclose(L, want2[:n, :n], rtol=0, atol=1e-12 * np.abs(want2).max())


def _manufactured(n, seed):
    """u of degree <= n - 1 in each variable (so that f and the solution fit the
    sizes the input and output maps take); returns U ((n+2) x (n+2))."""
    rng = np.random.default_rng(seed)
    m = n + 2
    U = np.zeros((m, m))
    U[:n, :n] = rng.standard_normal((n, n)) / np.add.outer(np.arange(n) + 1.0, np.arange(n) + 1.0)
    return U


@pytest.mark.parametrize("w,h", RECTS)
@pytest.mark.parametrize("n", [3, 12, 40])
def test_manufactured_polynomial_solution(n, w, h):
    kx, ky = oracle.rect_scales(w, h)
    U = _manufactured(n, 11 + n)
    G = laplacian_by_quadrature(U, kx, ky)[:n, :n]
    got = odir.poisson_dirichlet(G, traces(U), w, h, 1e-14)
    # f's coefficients grow like degree^2 (times the aspect ratio) against u's, so
    # rounding in f limits the recovered u to about that many ulps
    bar = 1e-14 * n * n * max(kx, ky) / min(kx, ky)
    assert np.abs(got - U).max() <= bar * np.abs(U).max()


def test_smooth_solution_converges_pointwise():
    """u = exp(x/2) sin(y + 0.3) + x^2 cosh(y) on a 3 x 1.5 rectangle (mapped to
    [-1,1]^2): f and the traces projected by Gauss-Legendre quadrature, the result
    evaluated at interior points against u itself."""
    w, h = 3.0, 1.5
    kx, ky = oracle.rect_scales(w, h)
    u = lambda x, y: np.exp(x / 2) * np.sin(y + 0.3) + x * x * np.cosh(y)
    f = lambda x, y: (kx * 0.25 * np.exp(x / 2) * np.sin(y + 0.3) + kx * 2 * np.cosh(y)
                      - ky * np.exp(x / 2) * np.sin(y + 0.3) + ky * x * x * np.cosh(y))
    xq, wq = npleg.leggauss(80)
    pts = np.random.default_rng(2).uniform(-0.95, 0.95, (2, 50))
    errs = []
    for n in (6, 9, 22):
        m = n + 2
        Pn = npleg.legvander(xq, n - 1) * (2 * np.arange(n) + 1) / 2.0   # projection weights
        Pm = npleg.legvander(xq, m - 1) * (2 * np.arange(m) + 1) / 2.0
        Y, X = np.meshgrid(xq, xq, indexing="ij")
        G = (Pn * wq[:, None]).T @ f(X, Y) @ (Pn * wq[:, None])
        one = np.ones_like(xq)
        bc = np.stack([(Pm * wq[:, None]).T @ u(-one, xq), (Pm * wq[:, None]).T @ u(one, xq),
                       (Pm * wq[:, None]).T @ u(xq, -one), (Pm * wq[:, None]).T @ u(xq, one)])
        Uc = odir.poisson_dirichlet(G, bc, w, h, 1e-14)
        errs.append(np.abs(npleg.legval2d(pts[1], pts[0], Uc) - u(pts[0], pts[1])).max())
    assert errs[0] > 10 * errs[1] and errs[1] > 10 * errs[2] and errs[2] < 1e-12, errs


def _dot(a, b):
    return float(np.sum(np.asarray(a) * np.asarray(b)))


@pytest.mark.parametrize("n", [1, 2, 7, 30])
def test_legendre_adjoints_are_transposes(n):
    rng = np.random.default_rng(n)
    G, Fb = rng.standard_normal((2, n, n))
    lhs = _dot(oracle.legendre_to_ctilde(G), Fb)
    assert abs(lhs - _dot(G, oracle.legendre_to_ctilde_adjoint(Fb))) <= 1e-13 * (1 + abs(lhs)) * n
    X = rng.standard_normal((n, n))
    Ub = rng.standard_normal((n + 2, n + 2))
    lhs = _dot(oracle.solution_to_legendre(X), Ub)
    assert abs(lhs - _dot(X, oracle.solution_to_legendre_adjoint(Ub))) <= 1e-12 * (1 + abs(lhs)) * n


@pytest.mark.parametrize("w,h", RECTS)
@pytest.mark.parametrize("n", [1, 4, 20])
def test_dirichlet_adjoint_dot_product(n, w, h):
    rng = np.random.default_rng(100 + n)
    G = rng.standard_normal((n, n))
    bc = rng.standard_normal((4, n + 2))      # need not agree at the corners: the map is linear anyway
    Ub = rng.standard_normal((n + 2, n + 2))
    U = odir.poisson_dirichlet(G, bc, w, h, 1e-14)
    Gb, bcb = odir.poisson_dirichlet_adjoint(Ub, w, h, 1e-14)
    lhs, rhs = _dot(U, Ub), _dot(G, Gb) + _dot(bc, bcb)
    scale = np.abs(U).max() * np.abs(Ub).sum()
    assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs)


def test_dirichlet_adjoint_against_exhaustive_jacobian():
    """n = 3 (m = 5): every column of the Jacobian of the linear map (G, bc) -> U by a
    forward solve of a unit input; the adjoint must equal J^T Ubar."""
    n, m = 3, 5
    w, h = 3.0, 0.75
    Ub = np.random.default_rng(9).standard_normal((m, m))
    Gb, bcb = odir.poisson_dirichlet_adjoint(Ub, w, h, 1e-15)
    zG, zb = np.zeros((n, n)), np.zeros((4, m))
    for a in range(n):
        for b in range(n):
            E = zG.copy()
            E[a, b] = 1.0
            col = odir.poisson_dirichlet(E, zb, w, h, 1e-15)
            assert abs(_dot(col, Ub) - Gb[a, b]) <= 1e-12 * max(1.0, abs(Gb[a, b]))
    for s in range(4):
        for k in range(m):
            E = zb.copy()
            E[s, k] = 1.0
            col = odir.poisson_dirichlet(zG, E, w, h, 1e-15)
            assert abs(_dot(col, Ub) - bcb[s, k]) <= 1e-12 * max(1.0, abs(bcb[s, k])), (s, k)
