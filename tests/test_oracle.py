"""Pins of the CPU oracle against facts the paper and the mathematics fix.

None of these re-types the oracle's own formulas: every expected value comes
from an independent route (Gauss quadrature of the basis, a dense Kronecker
solve, a closed-form DST solution, mpmath elliptic functions, a manufactured
polynomial solution, values printed in the paper)."""
import numpy as np
import pytest
import scipy.linalg
from scipy.fft import dst
from scipy.special import gegenbauer

import oracle
from oracle import basis
from paper_1710_11259_gb300 import inputs


def _dense_from_bands(d, e, s=2):
    n = len(d)
    A = np.diag(np.asarray(d, dtype=float))
    for j in range(n - s):
        A[j, j + s] = A[j + s, j] = e[j]
    return A


def _relmax(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


# ---------------------------------------------------------------- basis, M, D
@pytest.mark.parametrize("n", [1, 2, 7, 24])
def test_M_matches_quadrature(n):
    """(3.7) against Gauss-Jacobi quadrature of (1-x^2) C~_i C~_j (1-x^2)."""
    x, w = basis.gauss_jacobi(n + 8)
    B = basis.basis_matrix(n, x)
    Mq = (B * (w * (1 - x**2))) @ B.T
    d, e = oracle.M_bands(n)
    Mo = _dense_from_bands(d, e, 2)
    assert np.abs(Mo - Mq).max() < 1e-14
    # M_{j,j+1} = 0 and the band structure
    assert np.abs(np.triu(Mq, 3)).max() < 1e-14
    if n > 1:
        assert np.abs(np.diag(Mq, 1)).max() < 1e-14


def test_basis_orthonormal():
    """Footnote of Sec. 3.1: int C~_i C~_j (1-x^2) dx = delta_ij."""
    n = 30
    x, w = basis.gauss_jacobi(n + 2)
    B = basis.basis_matrix(n, x)
    G = (B * w) @ B.T
    assert np.abs(G - np.eye(n)).max() < 1e-13


@pytest.mark.parametrize("j", [0, 1, 2, 5, 11])
def test_eigen_identity(j):
    """(3.4): d^2/dx^2 [(1-x^2) C~_j] = -(j(j+3)+2) C~_j, checked as polynomials."""
    c = np.poly1d(gegenbauer(j, 1.5).coeffs)
    u = np.poly1d([-1.0, 0.0, 1.0]) * c
    lhs = u.deriv(2)
    rhs = -(j * (j + 3) + 2) * c
    x = np.linspace(-1, 1, 17)
    assert np.abs(lhs(x) - rhs(x)).max() <= 1e-9 * max(1.0, np.abs(rhs(x)).max())


def test_n1_special_case():
    """Proof of Lemma B.2: for n = 1, A~ = -2/5; so M X D + D X M = F gives X = -5F/16."""
    d, _ = oracle.square_bands(1)
    assert abs(d[0] - (-2.0 / 5.0)) < 1e-16
    F = np.array([[0.7]])
    X = oracle.poisson_square(F, 1e-13)
    assert abs(X[0, 0] - (-5.0 / 16.0) * 0.7) < 1e-13 * 0.7 * 5 / 16


@pytest.mark.parametrize("n", [2, 3, 8, 33, 128, 400])
def test_spectral_interval_lemma_B2(n):
    """Lemma B.2: sigma(A~) in [-1, -1/(30 n^4)]; the proof's sharper bound
    lambda_max < -3/(64 n^4) + 1/(64 n^5) as well."""
    d, e = oracle.square_bands(n)
    lam = np.linalg.eigvalsh(_dense_from_bands(d, e))
    assert lam.min() > -1.0
    assert lam.max() < -1.0 / (30.0 * n**4)
    assert lam.max() < -3.0 / (64.0 * n**4) + 1.0 / (64.0 * n**5)


def test_bands_symmetrise_A():
    """(3.9): A~ = D_s^{-1} (D^{-1} M) D_s is symmetric and similar to D^{-1} M."""
    n = 12
    d, e = oracle.M_bands(n)
    M = _dense_from_bands(d, e)
    Dm = np.diag([-(j * (j + 3) + 2.0) for j in range(n)])
    A = np.linalg.solve(Dm, M)
    ad, ae = oracle.square_bands(n)
    At = _dense_from_bands(ad, ae)
    assert np.abs(At - At.T).max() == 0.0
    assert np.allclose(np.sort(np.linalg.eigvals(A).real), np.sort(np.linalg.eigvalsh(At)), rtol=1e-12, atol=0)


# ----------------------------------------------------------- shifts, J
def _mobius_by_cross_ratio(alpha, a, b, c):
    """Independent construction of T: the cross-ratio of (w; a, b, c) equals that of
    (z; -alpha, -1, 1).  Returns w(z) as an mpmath function."""
    import mpmath as mp

    def T(z):
        s = (z + alpha) * (-1 - 1) / ((z - 1) * (-1 + alpha))
        # solve s = (w-a)(b-c)/((w-c)(b-a)) for w
        return (s * c * (b - a) - a * (b - c)) / (s * (b - a) - (b - c))
    return T


@pytest.mark.parametrize(
    "interval",
    [
        "square32", "square1000", "square10000",   # alpha >= 1e7: asymptotic branch
        "fd64",                                    # alpha = 4096: AGM branch
        "asym",                                    # non-symmetric intervals: general Moebius map
    ],
)
def test_shifts_against_mpmath(interval):
    """(2.4) against mpmath elliptic functions at 60 digits."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    if interval.startswith("square"):
        n = int(interval[6:])
        a, b, c, d = oracle.square_interval(n)
    elif interval == "fd64":
        a, b, c, d = -64.0**2, -1.0, 1.0, 64.0**2
    else:
        eps2 = 1e-10
        a, b, c, d = -1.0, -eps2, 2 * eps2, 2.0
    tol = 1e-13
    p, q = oracle.adi_shifts(a, b, c, d, tol)
    J = len(p)
    A, B, C, D = (mp.mpf(v) for v in (a, b, c, d))
    gam = abs(C - A) * abs(D - B) / (abs(C - B) * abs(D - A))
    alp = -1 + 2 * gam + 2 * mp.sqrt(gam**2 - gam)
    m = 1 - 1 / alp**2
    K = mp.ellipk(m)
    T = _mobius_by_cross_ratio(alp, A, B, C)
    assert abs(T(alp) - D) < mp.mpf(10) ** -20 * (1 + abs(D))
    for j in range(J):
        dn = mp.ellipfun("dn", (j + mp.mpf(1) / 2) * K / J, m=m)
        pj, qj = T(-alp * dn), T(alp * dn)
        assert abs(p[j] - pj) <= 1e-12 * abs(pj)
        assert abs(q[j] - qj) <= 1e-12 * abs(qj)
        assert a <= p[j] <= b and c <= q[j] <= d


def test_square_shifts_symmetric():
    """Symmetric intervals give alpha = 1/eps exactly and p_j = -q_j."""
    a, b, c, d = oracle.square_interval(256)
    p, q = oracle.adi_shifts(a, b, c, d, 1e-13)
    assert np.abs(p + q).max() <= 1e-15 * np.abs(q).max()


def _square_exact_Y(n, Ft):
    d, e = oracle.square_bands(n)
    At = _dense_from_bands(d, e)
    return scipy.linalg.solve_sylvester(At, At, Ft), d, e


@pytest.mark.parametrize("J", [2, 4, 8, 12, 16, 24])
def test_zolotarev_bound(J):
    """Theorem 2.1 with the simplified bound (2.6): ||Y - Y_J||_2 <= 4 exp(pi^2/(2 log 16 gamma))^{-2J} ||Y||_2."""
    n = 24
    Ft = inputs.square_rhs(n, 11, power=1)
    Y, d, e = _square_exact_Y(n, Ft)
    a, b, c, dd = oracle.square_interval(n)
    p, q = oracle.adi_shifts(a, b, c, dd, 0.5, J=J)
    YJ = oracle.adi_sylvester(2, d, e, -d, -e, Ft, p, q)
    gam = (c - a) * (dd - b) / ((c - b) * (dd - a))
    bound = 4.0 * np.exp(np.pi**2 / (2.0 * np.log(16.0 * gam))) ** (-2 * J)
    err = np.linalg.norm(Y - YJ, 2) / np.linalg.norm(Y, 2)
    assert err <= max(bound, 1e-14)


@pytest.mark.parametrize("tol", [1e-3, 1e-6, 1e-9, 1e-12])
def test_iteration_count_meets_tolerance(tol):
    """(2.9): with J = ceil(log(16 gamma) log(4/eps)/pi^2), ||Y - Y_J||_2 <= eps ||Y||_2."""
    n = 32
    Ft = inputs.square_rhs(n, 12, power=1)
    Y, d, e = _square_exact_Y(n, Ft)
    a, b, c, dd = oracle.square_interval(n)
    p, q = oracle.adi_shifts(a, b, c, dd, tol)
    YJ = oracle.adi_sylvester(2, d, e, -d, -e, Ft, p, q)
    err = np.linalg.norm(Y - YJ, 2) / np.linalg.norm(Y, 2)
    assert err <= max(tol, 5e-14)


# ----------------------------------------------------------- whole solver
@pytest.mark.parametrize("n", [2, 3, 5, 8, 17, 32])
def test_square_dense_kronecker(n):
    """(3.6) M X D^T + D X M^T = F solved densely (Kronecker form) vs the ADI solver."""
    d, e = oracle.M_bands(n)
    M = _dense_from_bands(d, e)
    Dm = np.diag([-(j * (j + 3) + 2.0) for j in range(n)])
    F = inputs.square_rhs(n, 0)
    L = np.kron(M, Dm) + np.kron(Dm, M)        # row-major vec: (M X D)_{ik} = sum M_ij X_jl D_lk
    Xd = np.linalg.solve(L, F.ravel()).reshape(n, n)
    X = oracle.poisson_square(F, 1e-13)
    assert _relmax(X, Xd) < 2e-13


@pytest.mark.parametrize("n", [16, 64])
def test_square_manufactured_polynomial(n):
    """u = (1-x^2)(1-y^2) p(x,y), deg p <= 10: the coefficients of p are recovered."""
    pc = basis.monomial_coeffs(inputs.poly_values(1), 10)
    F, Xe = basis.manufactured_square(pc, n)
    X = oracle.poisson_square(F, 1e-13)
    assert _relmax(X, Xe) < 2e-13


@pytest.mark.parametrize("n", [16, 64])
def test_fd_closed_form(n):
    """Sec. 2.1: ADI on K X + X K^T = F (1.2) with intervals [-n^2,-1], [1,n^2]
    against the DST-I closed form (1.3)."""
    m, h = n - 1, 2.0 / n
    Kd, Ke = np.full(m, -2 / h**2), np.full(m - 1, 1 / h**2)
    F = inputs.gaussian(3, (m, m))
    p, q = oracle.adi_shifts(-float(n) ** 2, -1.0, 1.0, float(n) ** 2, 1e-13)
    X = oracle.adi_sylvester(1, Kd, Ke, -Kd, -Ke, F, p, q)
    lam = -4 / h**2 * np.sin(np.pi * np.arange(1, n) / (2 * n)) ** 2
    S = lambda A: dst(dst(A, type=1, norm="ortho", axis=0), type=1, norm="ortho", axis=1)  # noqa: E731
    Xc = S(S(F) / (lam[:, None] + lam[None, :]))
    assert _relmax(X, Xc) < 1e-12


def test_solve_map_self_adjoint():
    """The map F -> X is a rational function of commuting symmetric operators
    (after the diagonal scalings of (3.9)), hence self-adjoint:  <P a, b> = <a, P b>."""
    n = 20
    a = inputs.gaussian(21, (n, n))
    b = inputs.gaussian(22, (n, n))
    Pa = oracle.poisson_square(a, 1e-13)
    Pb = oracle.poisson_square(b, 1e-13)
    lhs, rhs = np.vdot(Pa, b), np.vdot(a, Pb)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_longdouble_rounding_check():
    """The double oracle agrees with the long-double build of the same source."""
    if oracle.real_bytes("longdouble") <= 8:
        pytest.skip("long double is double on this platform")
    n = 96
    F = inputs.square_rhs(n, 2)
    X64 = oracle.poisson_square(F, 1e-13)
    Xld = oracle.poisson_square(F, 1e-13, variant="longdouble")
    assert _relmax(X64, Xld) < 1e-13


def test_golden_paper_values():
    """Values printed in the paper (tests/golden/paper_values.txt)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")
    vals = {}
    for line in open(path):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split("=")
            vals[k.strip()] = float(v)
    d, _ = oracle.square_bands(1)
    assert abs(d[0] - vals["A_tilde_n1"]) < 1e-16
    # D_jj = -(j(j+3)+2) enters through E; eigen-identity values for j = 0..3
    for j in range(4):
        assert vals[f"eig_identity_{j}"] == -(j * (j + 3) + 2)


# ----------------------------------------------------------- the cube (Sec. 5)
def _dense_cube_operator(n):
    d, e = oracle.M_bands(n)
    M = _dense_from_bands(d, e)
    Dm = np.diag([-(j * (j + 3) + 2.0) for j in range(n)])
    return np.kron(np.kron(Dm, M), M) + np.kron(np.kron(M, Dm), M) + np.kron(np.kron(M, M), Dm)


@pytest.mark.parametrize("n", [2, 3, 5])
def test_cube_dense_kronecker(n):
    """(5.2): the nested ADI of Sec. 5 against a dense solve of the Kronecker system."""
    F = inputs.cube_rhs(n, 6)
    Xd = np.linalg.solve(_dense_cube_operator(n), F.ravel()).reshape(n, n, n)
    X, J, inner = oracle.poisson_cube(F, 1e-13)
    assert J > 0 and inner > 0
    assert _relmax(X, Xd) < 5e-13


def test_cube_n1_closed_form():
    """n = 1: (D (x) M (x) M + ...) = 3 (-2)(4/5)^2 = -96/25, so X = -25 F / 96."""
    F = np.full((1, 1, 1), 0.3)
    X, _, _ = oracle.poisson_cube(F, 1e-13)
    assert abs(X[0, 0, 0] - (-25.0 / 96.0) * 0.3) <= 1e-12 * 0.3 * 25 / 96


def test_cube_manufactured_polynomial():
    """u = (1-x^2)(1-y^2)(1-z^2) p, deg p <= 2 in each variable: coefficients recovered."""
    n = 6
    pc = inputs.gaussian(13, (3, 3, 3))
    F, Xe = basis.manufactured_cube(pc, n)
    X, _, _ = oracle.poisson_cube(F, 1e-13)
    assert _relmax(X, Xe) < 5e-13


# ------------------------------------------- Legendre in / Legendre out (Sec. 3.4)
def _legendre_coeffs_2d(f, n, N):
    """c_ab with f = sum c_ab P_a(y) P_b(x), by Gauss-Legendre quadrature (exact for
    polynomials of degree < 2N - n in each variable)."""
    x, w = np.polynomial.legendre.leggauss(N)
    P = np.stack([np.polynomial.legendre.legval(x, np.eye(n)[a]) for a in range(n)])  # [a, node]
    Xg, Yg = np.meshgrid(x, x, indexing="xy")  # Xg[iy, ix] = x[ix]
    vals = f(Xg, Yg)
    scale = (2 * np.arange(n) + 1) / 2.0
    return (scale[:, None] * (P * w)) @ vals @ (scale[:, None] * (P * w)).T


@pytest.mark.parametrize("n", [1, 2, 5, 12])
def test_legendre_to_ctilde_against_quadrature(n):
    """F = B G B^T equals the C~ projection (Gauss-Jacobi quadrature) of sum G P_a(y) P_b(x)."""
    G = inputs.gaussian(21, (n, n))
    f = lambda X, Y: np.polynomial.legendre.legval2d(Y, X, G)
    Fq = basis.project_2d(f, n, n + 4)
    assert np.abs(oracle.legendre_to_ctilde(G) - Fq).max() <= 1e-13 * np.abs(Fq).max()


@pytest.mark.parametrize("n", [1, 3, 10])
def test_solution_to_legendre_pointwise(n):
    """The Legendre series U reproduces u = (1-x^2)(1-y^2) sum X_ij C~_i(y) C~_j(x) at points."""
    X = inputs.gaussian(22, (n, n))
    U = oracle.solution_to_legendre(X)
    pts = np.linspace(-0.97, 0.99, 9)
    xs, ys = np.meshgrid(pts, pts)
    Cx = basis.basis_matrix(n, xs.ravel())  # [j, point]
    Cy = basis.basis_matrix(n, ys.ravel())
    u = (1 - xs.ravel() ** 2) * (1 - ys.ravel() ** 2) * np.einsum("ip,ij,jp->p", Cy, X, Cx)
    ul = np.polynomial.legendre.legval2d(ys.ravel(), xs.ravel(), U)
    assert np.abs(u - ul).max() <= 1e-13 * np.abs(u).max()


def test_legendre_roundtrip_manufactured():
    """Legendre coefficients of f = Laplacian(u) in, solve (3.6), Legendre coefficients of
    u = (1-x^2)(1-y^2) p out, against u's own coefficients (deg p <= 6, n = 16)."""
    n = 16
    pc = basis.monomial_coeffs(inputs.gaussian(23, (28,)), 6)
    uc = basis.poly_times_bubble(pc)
    fc = basis.laplacian(uc)
    G = _legendre_coeffs_2d(lambda X, Y: basis.poly_eval(fc, X, Y), n, n + 8)
    X = oracle.poisson_square(oracle.legendre_to_ctilde(G), 1e-13)
    U = oracle.solution_to_legendre(X)
    Ue = _legendre_coeffs_2d(lambda X, Y: basis.poly_eval(uc, X, Y), n + 2, n + 10)
    assert np.abs(U - Ue).max() <= 1e-12 * np.abs(Ue).max()


def test_cube_spectral_convergence_fig51():
    """The cube discretisation converges spectrally to the true solution: for the
    function of Fig. 5.1, u = (1-x^2)(1-y^2)(1-z^2) cos(x y z^2), the computed
    coefficients approach the C~ coefficients of cos(x y z^2) (the ansatz (3.2) in
    three variables) by orders of magnitude as n grows."""
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    u = (1 - x**2) * (1 - y**2) * (1 - z**2) * sp.cos(x * y * z**2)
    f = sp.lambdify((x, y, z), sp.diff(u, x, 2) + sp.diff(u, y, 2) + sp.diff(u, z, 2), "numpy")
    p = sp.lambdify((x, y, z), sp.cos(x * y * z**2), "numpy")
    errs = []
    for n in (4, 8, 12):
        F = basis.project_3d(f, n, n + 24)
        Xe = basis.project_3d(p, n, n + 24)
        X, _, _ = oracle.poisson_cube(F, 1e-11, 1e-13, 1e-13)
        errs.append(np.abs(X - Xe).max())
    assert errs[0] > 1e2 * errs[1] > 1e4 * errs[2]
    assert errs[2] < 1e-8


# ------------------------------------------------- tight spectral interval (f1)
@pytest.mark.parametrize("n", [1, 2, 3, 10, 64, 300])
def test_tight_interval_contains_spectrum(n):
    """The oracle's Sturm-bisection interval contains sigma(A~) (eigvalsh) with the
    stated padding: lo = |lambda_max| / 2, hi = min(1, 1.01 |lambda_min|)."""
    lo, hi = oracle.tight_interval(n)
    d, e = oracle.square_bands(n)
    lam = np.linalg.eigvalsh(_dense_from_bands(d, e))
    small, big = -lam.max(), -lam.min()
    assert lo <= small and hi >= big
    assert abs(lo - 0.5 * small) <= 1e-9 * small
    assert abs(hi - min(1.0, 1.01 * big)) <= 1e-12


@pytest.mark.parametrize("n", [1, 2, 3, 10, 64, 300, 2048, 10000])
def test_tight_interval_library_agrees_with_oracle(n):
    """The library's own bisection (host helper) and the oracle's give the same interval
    and therefore the same J of (2.9) (133 -> 110 at n = 10^4, tol 1e-13)."""
    from paper_1710_11259_gb300 import api

    a = oracle.tight_interval(n)
    b = api.square_spectral_interval(n, True)
    assert abs(a[0] - b[0]) <= 1e-9 * a[0] and abs(a[1] - b[1]) <= 1e-12 * a[1]
    Ja = oracle.adi_iterations(-a[1], -a[0], a[0], a[1], 1e-13)
    Jb = oracle.adi_iterations(-b[1], -b[0], b[0], b[1], 1e-13)
    assert Ja == Jb <= oracle.square_iterations(n, 1e-13)


@pytest.mark.parametrize("n", [10, 64, 300, 10000])
def test_tight_interval_shifts_against_mpmath(n):
    """Shifts of the tight interval: q_j = hi dn((2j+1)K/(2J); k' = lo/hi) computed with
    mpmath at 40 digits.  The library (complementary-modulus route) is exact to 1e-10;
    the oracle follows App. A, whose alpha < 1e7 branch forms m = 1 - 1/alpha^2 in FP64
    and so keeps only about ten digits less than that (6e-7 at n = 64, alpha ~ 4e5)."""
    mpmath = pytest.importorskip("mpmath")
    from paper_1710_11259_gb300 import api

    mpmath.mp.dps = 40
    lo, hi = oracle.tight_interval(n)
    J = oracle.adi_iterations(-hi, -lo, lo, hi, 1e-13)
    kp = mpmath.mpf(lo) / mpmath.mpf(hi)
    m = 1 - kp**2
    K = mpmath.ellipk(m)
    exact = np.array([float(hi * mpmath.ellipfun("dn", (2 * j + 1) * K / (2 * J), m=m)) for j in range(J)])
    _, ql = api.zolotarev_shifts(-hi, -lo, lo, hi, 1e-13, J)
    _, qo = oracle.adi_shifts(-hi, -lo, lo, hi, 1e-13, J)
    rel = lambda a: float(np.max(np.abs(np.sort(a) - np.sort(exact)) / np.sort(exact)))
    assert rel(ql) <= 1e-10
    assert rel(qo) <= 2e-6


# ------------------------------------------------------------ rectangle (f2)
@pytest.mark.parametrize("n,w,h", [(3, 2.0, 0.5), (8, 1.0, 3.0), (17, 5.0, 2.0)])
def test_rectangle_dense_kronecker(n, w, h):
    """kx M X D^T + ky D X M^T = F (the rectangle form of (3.6)) solved densely."""
    kx, ky = oracle.rect_scales(w, h)
    d, e = oracle.M_bands(n)
    M = _dense_from_bands(d, e)
    Dm = np.diag([-(j + 1.0) * (j + 2.0) for j in range(n)])
    F = inputs.square_rhs(n, 5)
    L = kx * np.kron(M, Dm) + ky * np.kron(Dm, M)
    Xd = np.linalg.solve(L, F.ravel()).reshape(n, n)
    X, J = oracle.poisson_rectangle(F, w, h, 1e-13)
    assert _relmax(X, Xd) < 2e-13
    assert J > 0


def test_rectangle_reduces_to_square():
    F = inputs.square_rhs(40, 6)
    X, _ = oracle.poisson_rectangle(F, 2.0, 2.0, 1e-13)
    assert np.array_equal(X, oracle.poisson_square(F, 1e-13))


@pytest.mark.parametrize("w,h", [(2.0, 0.5), (6.0, 1.5)])
def test_rectangle_manufactured(w, h):
    """u = (1-s^2)(1-t^2) p(s,t) on a w x h rectangle (deg p = 10): coefficients recovered."""
    kx, ky = oracle.rect_scales(w, h)
    pc = basis.monomial_coeffs(inputs.poly_values(1), 10)
    F, Xe = basis.manufactured_rectangle(pc, 32, kx, ky)
    X, _ = oracle.poisson_rectangle(F, w, h, 1e-13)
    assert _relmax(X, Xe) < 5e-13
