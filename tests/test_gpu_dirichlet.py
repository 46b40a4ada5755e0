"""GPU parity of the nonhomogeneous Dirichlet solve (Sec. 6.1) and its adjoint through
the C ABI: against the CPU oracle element by element (the solve's parity bar, FP64
1e-12 and refined 1e-10 of max|X|, carried entry by entry through the output map
U = L X L^T, whose row gains grow like sqrt(degree)), a manufactured polynomial solution
at n = 4096, the dot-product identity of the adjoint at n = 4096, central
differences of a quadratic loss in the boundary traces and the right-hand side, and
torch.autograd.gradcheck."""
import numpy as np
import pytest

import oracle
from oracle import dirichlet as odir
from dirichlet_helpers import laplacian_by_quadrature, traces
from paper_1710_11259_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SQUARE = (2.0, 2.0)


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_11259_gb300 import api as _api
    from paper_1710_11259_gb300 import build_ext

    build_ext.build()
    _api.lib()
    return _api


def _relmax(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _out_gain(n):
    """l_i = c_i + c_{i-2} (i < n + 2): the absolute row sums of the output map
    U = L X L^T (L[j][j] = c_j, L[j+2][j] = -c_j, c_j = s_j (j+1)(j+2)/(2j+3)), so an
    error e in X moves U[i][j] by at most e l_i l_j."""
    j = np.arange(n, dtype=np.float64)
    c = np.sqrt((j + 1.5) / ((j + 1) * (j + 2))) * (j + 1) * (j + 2) / (2 * j + 3)
    ell = np.zeros(n + 2)
    ell[:n] += c
    ell[2:] += c
    return ell


def _oracle_solution(G, bc, wh, tol=1e-13):
    """The oracle's U and the largest coefficient of its homogeneous solution X."""
    kx, ky = oracle.rect_scales(*wh)
    F = oracle.legendre_to_ctilde(G - odir.lift_laplacian(bc, kx, ky))
    if wh == SQUARE:
        X = oracle.poisson_square(F, tol)
    else:
        X = oracle.poisson_rectangle(F, wh[0], wh[1], tol)[0]
    return oracle.solution_to_legendre(X) + odir.lift(bc), float(np.abs(X).max())


def _check_U(U, G, bc, wh, bar):
    """Entry by entry: the solve's parity bar (bar x max|X|) carried through the output
    map, plus bar x 0.1 of max|U| for the O(n) lifting and Laplacian steps."""
    Uo, xmax = _oracle_solution(G, bc, wh)
    ell = _out_gain(G.shape[-1])
    allowed = bar * xmax * np.outer(ell, ell) + 0.1 * bar * np.abs(Uo).max()
    worst = float((np.abs(U - Uo) / allowed).max())
    assert worst <= 1.0, worst
    return Uo


def _plan(api, n, wh, tol, precision, nrhs=1):
    if wh == SQUARE:
        return api.plan_create(n, 2, tol, precision, nrhs=nrhs)
    return api.plan_create_rect(n, wh[0], wh[1], tol, precision, nrhs=nrhs)


def _data(n, seed, lead=()):
    """Right-hand side and traces with decaying coefficients; the traces need not agree
    at the corners (the corner value is then the mean of the two meeting traces).  The
    traces' coefficients fall like k^-4 (twice-differentiable data, so g'' has bounded
    coefficients): with rougher traces lap u_bc grows like k^2 times them and dominates
    the right-hand side, and any comparison then measures the rounding of that sum."""
    m = n + 2
    G = inputs.gaussian(seed, lead + (n, n)) / np.add.outer(np.arange(n) + 1.0, np.arange(n) + 1.0) ** 2
    bc = inputs.gaussian(seed + 1, lead + (4, m)) / (np.arange(m) + 1.0) ** 4
    return np.ascontiguousarray(G), np.ascontiguousarray(bc)


def _solve(api, plan, G, bc):
    U = api.poisson_dirichlet_solve(plan, torch.from_numpy(G).cuda(), torch.from_numpy(bc).cuda())
    return U.cpu().numpy()


@pytest.mark.parametrize("wh", [SQUARE, (3.0, 0.75)])
@pytest.mark.parametrize("n", [1, 2, 3, 17, 64, 65, 300, 1000])
def test_dirichlet_fp64_matches_oracle(api, n, wh):
    G, bc = _data(n, 10 + n)
    plan = _plan(api, n, wh, 1e-13, "fp64")
    U = _solve(api, plan, G, bc)
    api.plan_destroy(plan)
    _check_U(U, G, bc, wh, 1e-12)


@pytest.mark.parametrize("n,wh", [(33, SQUARE), (300, (1.0, 3.0)), (1000, (5.0, 2.0))])
def test_dirichlet_refined_matches_oracle(api, n, wh):
    G, bc = _data(n, 30 + n)
    plan = _plan(api, n, wh, 1e-10, "fp32_refine")
    U = _solve(api, plan, G, bc)
    api.plan_destroy(plan)
    _check_U(U, G, bc, wh, 1e-10)


def test_dirichlet_two_right_hand_sides(api):
    n, wh = 100, (3.0, 0.75)
    G, bc = _data(n, 7, (2,))
    plan = _plan(api, n, wh, 1e-13, "fp64", nrhs=2)
    U = _solve(api, plan, G, bc)
    api.plan_destroy(plan)
    for r in range(2):
        _check_U(U[r], G[r], bc[r], wh, 1e-12)


@pytest.mark.parametrize("precision,bar", [("fp64", 1e-11), ("fp32_refine", 1e-9)])
def test_dirichlet_manufactured_polynomial_n4096(api, precision, bar):
    """u of degree 29 in each variable on a 4 x 1 rectangle, solved at n = 4096: the
    solution's coefficients come back (zero beyond degree 29)."""
    n, d, wh = 4096, 30, (4.0, 1.0)
    kx, ky = oracle.rect_scales(*wh)
    Us = np.zeros((d + 2, d + 2))
    Us[:d, :d] = inputs.gaussian(5, (d, d)) / np.add.outer(np.arange(d) + 1.0, np.arange(d) + 1.0)
    Gs = laplacian_by_quadrature(Us, kx, ky)[:d, :d]
    G = np.zeros((n, n))
    G[:d, :d] = Gs
    U_true = np.zeros((n + 2, n + 2))
    U_true[: d + 2, : d + 2] = Us
    bc = traces(U_true)
    plan = _plan(api, n, wh, 1e-13 if precision == "fp64" else 1e-10, precision)
    U = _solve(api, plan, G, bc)
    api.plan_destroy(plan)
    assert _relmax(U, U_true) <= bar


@pytest.mark.parametrize("wh", [SQUARE, (0.5, 4.0)])
@pytest.mark.parametrize("n", [1, 2, 17, 300])
def test_dirichlet_adjoint_matches_oracle(api, n, wh):
    m = n + 2
    Ub = inputs.gaussian(50 + n, (m, m))
    plan = _plan(api, n, wh, 1e-13, "fp64")
    Gb, bcb = api.poisson_dirichlet_adjoint(plan, torch.from_numpy(Ub).cuda())
    api.plan_destroy(plan)
    Gbo, _ = odir.poisson_dirichlet_adjoint(Ub, wh[0], wh[1], 1e-13)
    Gb = Gb.cpu().numpy()
    assert _relmax(Gb, Gbo) <= 1e-12
    # the trace gradient applies D2^T (gains up to j^4/8) to rows and columns 0, 1 of
    # dL/dG, so it is compared stage by stage: against the oracle's trace step fed
    # with the library's own dL/dG, within 1e-12 of its largest entry plus the rounding
    # bound of the sums D2^T v (m eps sum_k |D2[k][j]| |v_k|: their terms cancel)
    ref = odir.traces_adjoint(Ub, Gb, wh[0], wh[1])
    kx, ky = oracle.rect_scales(*wh)
    D2 = np.abs(np.polynomial.legendre.legder(np.eye(m), 2, axis=0))       # (m-2) x m = n x m
    a0, a1 = np.abs(Gb[:, 0]), (np.abs(Gb[:, 1]) if n > 1 else 0 * Gb[:, 0])
    r0, r1 = np.abs(Gb[0, :]), (np.abs(Gb[1, :]) if n > 1 else 0 * Gb[0, :])
    v = np.stack([0.5 * ky * (a0 + a1)] * 2 + [0.5 * kx * (r0 + r1)] * 2)  # bounds of |v_side|
    cond = v @ D2
    allowed = 1e-12 * np.abs(ref).max() + m * 2.3e-16 * cond
    assert (np.abs(bcb.cpu().numpy() - ref) <= allowed).all()


@pytest.mark.parametrize("precision,bar", [("fp64", 1e-12), ("fp32_refine", 1e-9)])
def test_dirichlet_adjoint_dot_product_n4096(api, precision, bar):
    """<U(G, bc), Ubar> = <G, Gbar> + <bc, bcbar> for the library's own forward and
    adjoint maps at full size (the refined map is linear only to its tolerance)."""
    n, wh = 4096, (3.0, 1.2)
    G, bc = _data(n, 61)
    Ub = inputs.gaussian(62, (n + 2, n + 2)) / np.add.outer(np.arange(n + 2) + 1.0, np.arange(n + 2) + 1.0)
    plan = _plan(api, n, wh, 1e-13 if precision == "fp64" else 1e-11, precision)
    Gd, bd, Ubd = (torch.from_numpy(a).cuda() for a in (G, bc, Ub))
    U = api.poisson_dirichlet_solve(plan, Gd, bd)
    Gb, bcb = api.poisson_dirichlet_adjoint(plan, Ubd)
    api.plan_destroy(plan)
    lhs = float((U * Ubd).sum())
    rhs = float((Gd * Gb).sum() + (bd * bcb).sum())
    scale = float(U.abs().max() * Ubd.abs().sum())
    assert abs(lhs - rhs) <= bar * scale, (lhs, rhs)


def test_dirichlet_gradient_by_central_differences(api):
    """L = 0.5 ||U - U*||^2 is exactly quadratic in (G, bc): central differences along
    seeded unit directions in the traces and in G match the adjoint's gradient."""
    from paper_1710_11259_gb300 import autograd

    n, wh = 300, (3.0, 0.75)
    G, bc = _data(n, 71)
    Ustar = torch.from_numpy(inputs.gaussian(72, (n + 2, n + 2))).cuda()
    plan = _plan(api, n, wh, 1e-13, "fp64")
    Gt = torch.from_numpy(G).cuda().requires_grad_(True)
    bt = torch.from_numpy(bc).cuda().requires_grad_(True)
    loss = 0.5 * ((autograd.poisson_dirichlet(Gt, bt, plan) - Ustar) ** 2).sum()
    loss.backward()

    def L(Gv, bv):
        U = api.poisson_dirichlet_solve(plan, Gv, bv)
        return 0.5 * float(((U - Ustar) ** 2).sum())

    worst = 0.0
    for k in range(8):
        for which in ("bc", "G"):
            base = bt.detach() if which == "bc" else Gt.detach()
            d = torch.from_numpy(inputs.gaussian(80 + k, tuple(base.shape))).cuda()
            d /= d.norm()
            h = 1e-2 * float(base.norm())
            if which == "bc":
                fd = (L(Gt.detach(), base + h * d) - L(Gt.detach(), base - h * d)) / (2 * h)
                an = float((bt.grad * d).sum())
            else:
                fd = (L(base + h * d, bt.detach()) - L(base - h * d, bt.detach())) / (2 * h)
                an = float((Gt.grad * d).sum())
            gmax = float(max(bt.grad.abs().max(), Gt.grad.abs().max()))
            worst = max(worst, abs(fd - an) / gmax)
    api.plan_destroy(plan)
    assert worst <= 1e-6, worst


def test_dirichlet_gradcheck(api):
    from paper_1710_11259_gb300 import autograd

    n = 5
    plan = _plan(api, n, (3.0, 0.75), 1e-14, "fp64")
    G, bc = _data(n, 90)
    Gt = torch.from_numpy(G).cuda().requires_grad_(True)
    bt = torch.from_numpy(bc).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda a, b: autograd.poisson_dirichlet(a, b, plan), (Gt, bt), eps=1e-6,
                                    atol=1e-7, rtol=1e-6)
    api.plan_destroy(plan)


def test_dirichlet_rejects_host_buffers_and_batched_plans(api):
    import ctypes

    n = 8
    G, bc = _data(n, 3)
    plan = _plan(api, n, SQUARE, 1e-13, "fp64")
    with pytest.raises(api.FpsError) as e:
        api.poisson_dirichlet_solve(plan, torch.from_numpy(G), torch.from_numpy(bc).cuda(),
                                    torch.empty((n + 2, n + 2), dtype=torch.float64, device="cuda"))
    assert e.value.status == -1 and "device memory" in str(e.value)
    api.plan_destroy(plan)
    batch = api.plan_create_batched([8, 4], 1, 1e-10, "fp32_refine")
    Gd, bd = torch.from_numpy(G).cuda(), torch.from_numpy(bc).cuda()
    Ud = torch.empty((n + 2, n + 2), dtype=torch.float64, device="cuda")
    st = api.lib().fps_poisson_dirichlet_solve(batch.handle, ctypes.c_void_p(Gd.data_ptr()),
                                               ctypes.c_void_p(bd.data_ptr()), ctypes.c_void_p(Ud.data_ptr()))
    api.plan_destroy(batch)
    assert st == -1 and b"single square or rectangle" in api.lib().fps_last_error()
