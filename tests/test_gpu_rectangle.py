"""GPU parity of the rectangle solve (Sec. 3 on [x0, x0 + w] x [y0, y0 + h]): kx A~ Y + ky Y A~ = F~
with App. A's non-symmetric shifts, through the C ABI, against the CPU oracle (FP64 bar 1e-12,
refined bar 1e-10) and a manufactured polynomial solution."""
import numpy as np
import pytest

import oracle
from oracle import basis
from paper_1710_11259_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def _rect_solve(api, F, w, h, tol, precision):
    plan = api.plan_create_rect(F.shape[-1], w, h, tol, precision, nrhs=1 if F.ndim == 2 else F.shape[0])
    X = api.poisson_square_solve(plan, torch.from_numpy(F).cuda()).cpu().numpy()
    info = api.plan_info(plan)
    api.plan_destroy(plan)
    return X, info


@pytest.mark.parametrize("n,w,h", [(1, 2.0, 0.5), (33, 2.0, 0.5), (64, 1.0, 3.0), (100, 6.0, 1.5), (257, 0.3, 2.0),
                                   (1000, 4.0, 1.0)])
def test_rectangle_fp64_matches_oracle(api, n, w, h):
    F = inputs.square_rhs(n, 60 + n)
    X, info = _rect_solve(api, F, w, h, 1e-13, "fp64")
    Xo, J = oracle.poisson_rectangle(F, w, h, 1e-13)
    assert info["J"] == J
    assert _relmax(X, Xo) <= 1e-12


@pytest.mark.parametrize("n,w,h", [(33, 2.0, 0.5), (300, 1.0, 3.0), (2048, 5.0, 2.0)])
def test_rectangle_refined_matches_oracle(api, n, w, h):
    F = inputs.square_rhs(n, 80 + n)
    X, info = _rect_solve(api, F, w, h, 1e-10, "fp32_refine")
    Xo, _ = oracle.poisson_rectangle(F, w, h, 1e-13)
    assert info["last_residual"] <= 1e-10
    assert _relmax(X, Xo) <= 1e-10


def test_rectangle_square_limit_equals_square_plan(api):
    """A 2 x 2 rectangle is [-1,1]^2: the same shifts and the same result as the square plan."""
    n = 300
    F = torch.from_numpy(inputs.square_rhs(n, 5)).cuda()
    pr = api.plan_create_rect(n, 2.0, 2.0, 1e-13, "fp64")
    ps = api.plan_create(n, 2, 1e-13, "fp64")
    Xr = api.poisson_square_solve(pr, F)
    Xs = api.poisson_square_solve(ps, F)
    qr, qs = api.plan_shifts(pr), api.plan_shifts(ps)
    api.plan_destroy(pr)
    api.plan_destroy(ps)
    assert np.array_equal(qr, qs)
    assert torch.equal(Xr, Xs)


def test_rectangle_manufactured(api):
    """u = (1-s^2)(1-t^2) p(s,t) on a 6 x 1.5 rectangle, deg p = 10: coefficients recovered."""
    w, h = 6.0, 1.5
    kx, ky = oracle.rect_scales(w, h)
    F, Xe = basis.manufactured_rectangle(basis.monomial_coeffs(inputs.poly_values(1), 10), 80, kx, ky)
    X, _ = _rect_solve(api, F, w, h, 1e-13, "fp64")
    assert _relmax(X, Xe) <= 1e-12


def test_rectangle_adjoint_is_the_same_solve(api):
    """kx A~ + ky (.)A~ is self-adjoint, so dL/dF through fps_poisson_adjoint is the solve of dL/dX."""
    n = 200
    a = torch.from_numpy(inputs.gaussian(41, (n, n))).cuda()
    b = torch.from_numpy(inputs.gaussian(42, (n, n))).cuda()
    plan = api.plan_create_rect(n, 3.0, 0.7, 1e-13, "fp64")
    Pa = api.poisson_square_solve(plan, a)
    Pb = api.poisson_adjoint(plan, b)
    lhs, rhs = float((Pa * b).sum()), float((a * Pb).sum())
    scale = max(float(Pa.norm() * b.norm()), float(a.norm() * Pb.norm()))
    api.plan_destroy(plan)
    assert abs(lhs - rhs) <= 1e-13 * scale
