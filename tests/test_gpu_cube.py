"""GPU parity of the cube solve (nested ADI of Sec. 5, FP64) against the CPU oracle,
through the C ABI.  Tolerance: relative max-coefficient error <= 1e-12."""
import numpy as np
import pytest

import oracle
from oracle import basis
from paper_1710_11259_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-12


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


def _cube_solve(api, F, tol=1e-13):
    plan = api.plan_create(F.shape[-1], 3, tol, "fp64", nrhs=1 if F.ndim == 3 else F.shape[0])
    X = api.poisson_cube_solve(plan, torch.from_numpy(F).cuda())
    torch.cuda.synchronize()
    info = api.plan_info(plan)
    api.plan_destroy(plan)
    return X.cpu().numpy(), info


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_cube_matches_oracle(api, n):
    F = inputs.cube_rhs(n, 6)
    X, info = _cube_solve(api, F)
    Xo, J, _ = oracle.poisson_cube(F, 1e-13)
    assert info["J"] == J
    assert _relmax(X, Xo) <= TOL_FP64


def test_cube_manufactured(api):
    n = 6
    pc = inputs.gaussian(13, (3, 3, 3))
    F, Xe = basis.manufactured_cube(pc, n)
    X, _ = _cube_solve(api, F)
    assert _relmax(X, Xe) <= 5e-13


def _cube_by_diagonalisation(F):
    """Independent exact solve of (5.2): with A~ = V diag(lam) V^T (numpy eigh), the
    symmetrised operator T_01 + T_02 + T_12 is diagonal in V (x) V (x) V."""
    n = F.shape[0]
    d, e = oracle.square_bands(n)
    At = np.diag(d)
    for j in range(n - 2):
        At[j, j + 2] = At[j + 2, j] = e[j]
    lam, V = np.linalg.eigh(At)
    s = 1.0 / np.sqrt((np.arange(n) + 1.0) * (np.arange(n) + 2.0))
    S3 = s[:, None, None] * s[None, :, None] * s[None, None, :]
    G = -F * S3
    Gh = np.einsum("ai,bj,ck,abc->ijk", V, V, V, G)
    L = lam[:, None, None] * lam[None, :, None]
    den = L + lam[:, None, None] * lam[None, None, :] + lam[None, :, None] * lam[None, None, :]
    Yh = Gh / den
    Y = np.einsum("ia,jb,kc,abc->ijk", V, V, V, Yh)
    return Y * S3


@pytest.mark.parametrize("n", [17, 32])
def test_cube_against_diagonalisation(api, n):
    """Sizes the oracle cannot reach in seconds: against an exact solve by diagonalising A~."""
    F = inputs.cube_rhs(n, 6)
    X, info = _cube_solve(api, F)
    Xd = _cube_by_diagonalisation(F)
    assert _relmax(X, Xd) <= 1e-11


def test_cube_self_adjoint_and_host_path(api):
    n = 4
    a = inputs.gaussian(71, (n, n, n))
    b = inputs.gaussian(72, (n, n, n))
    plan = api.plan_create(n, 3, 1e-13, "fp64")
    Pa = api.poisson_cube_solve(plan, a)             # host arrays: staged by the library
    Pb = api.poisson_adjoint(plan, b)
    Pa_dev = api.poisson_cube_solve(plan, torch.from_numpy(a).cuda()).cpu().numpy()
    api.plan_destroy(plan)
    assert np.array_equal(Pa, Pa_dev)
    lhs, rhs = float(np.vdot(Pa, b)), float(np.vdot(a, Pb))
    # the nested map is self-adjoint up to the accuracy of its inner and middle
    # solves (each stopped at its tolerance): measured 1.1e-12 relative at n = 4
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)
