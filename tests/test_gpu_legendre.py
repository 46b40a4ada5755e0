"""GPU Legendre coefficients in and out (Sec. 3.4, Table 3.1 steps 1 and 4) through the
C ABI, against the oracle (which forms M X M^T and back-substitutes with B, a
different route from the kernel's two-term map) and end to end through a solve."""
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


@pytest.mark.parametrize("n", [1, 2, 5, 64, 257, 4096])
def test_conversions_match_oracle(api, n):
    G = inputs.gaussian(31, (n, n))
    X = inputs.square_rhs(n, 32)
    F = api.legendre_to_ctilde(torch.from_numpy(G).cuda())
    U = api.solution_to_legendre(torch.from_numpy(X).cuda())
    torch.cuda.synchronize()
    assert U.shape == (n + 2, n + 2)
    assert _relmax(F.cpu().numpy(), oracle.legendre_to_ctilde(G)) <= 1e-14
    assert _relmax(U.cpu().numpy(), oracle.solution_to_legendre(X)) <= 1e-13


def _legendre_coeffs_2d(f, n, N):
    x, w = np.polynomial.legendre.leggauss(N)
    P = np.stack([np.polynomial.legendre.legval(x, np.eye(n)[a]) for a in range(n)])
    Xg, Yg = np.meshgrid(x, x, indexing="xy")
    scale = (2 * np.arange(n) + 1) / 2.0
    return (scale[:, None] * (P * w)) @ f(Xg, Yg) @ (scale[:, None] * (P * w)).T


def test_legendre_round_trip_through_the_solve(api):
    """Legendre coefficients of f = Laplacian((1-x^2)(1-y^2) p) in, FP64 solve, Legendre
    coefficients of u out, against u's own (deg p <= 8, n = 24)."""
    n = 24
    pc = basis.monomial_coeffs(inputs.gaussian(33, (45,)), 8)
    uc = basis.poly_times_bubble(pc)
    fc = basis.laplacian(uc)
    G = _legendre_coeffs_2d(lambda X, Y: basis.poly_eval(fc, X, Y), n, n + 10)
    plan = api.plan_create(n, 2, 1e-13, "fp64")
    F = api.legendre_to_ctilde(torch.from_numpy(G).cuda())
    X = api.poisson_square_solve(plan, F)
    U = api.solution_to_legendre(X)
    torch.cuda.synchronize()
    api.plan_destroy(plan)
    Ue = _legendre_coeffs_2d(lambda X, Y: basis.poly_eval(uc, X, Y), n + 2, n + 12)
    assert _relmax(U.cpu().numpy(), Ue) <= 1e-12


def test_conversions_reject_host_memory(api):
    G = np.zeros((4, 4))
    with pytest.raises(api.FpsError) as e:
        api.legendre_to_ctilde(torch.from_numpy(G), torch.from_numpy(G.copy()))
    assert e.value.status == -1
