"""The allocation-free square solve (fps_poisson_square_solve_noalloc), called
through the C ABI, against the plan-based FP64 solve.

That entry point serves callers who cannot allocate device memory when they
solve: it keeps its work arrays in one fixed device array inside the library.
Two calls in a row with different right-hand sides check that the shared array's
leftover contents never reach a result.  This file is collected last so that a
run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

import oracle
from paper_1710_11259_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-12  # the FP64 parity bar used by the other GPU tests


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_11259_gb300 import api as _api
    from paper_1710_11259_gb300 import build_ext

    build_ext.build()
    _api.lib()
    return _api


def _plan_solve(api, F):
    plan = api.plan_create(F.shape[-1], 2, 1e-13, "fp64")
    X = api.poisson_square_solve(plan, F)
    torch.cuda.synchronize()
    api.plan_destroy(plan)
    return X


@pytest.mark.parametrize("n", [1, 2, 33, 100, 256])
def test_noalloc_matches_plan_solve_twice(api, n):
    for call, seed in enumerate((500 + n, 900 + n)):
        F = torch.from_numpy(inputs.square_rhs(n, seed)).cuda()
        X = torch.full_like(F, float("nan"))
        status = api.poisson_square_solve_noalloc(F, X, 1e-13)
        torch.cuda.synchronize()
        assert status == 0, f"call {call}: status {status}"
        Xp = _plan_solve(api, F)
        err = float((X - Xp).abs().max() / Xp.abs().max())
        assert err <= TOL_FP64, f"call {call}: rel-max diff {err:.3e}"


def test_noalloc_matches_oracle_n64(api):
    """Independent of the plan's kernels: the n = 64 right-hand side with decay
    1/((1+j)^2(1+k)^2) (seed 0) against the CPU oracle at the FP64 bar."""
    Fh = inputs.square_rhs(64, 0)
    F = torch.from_numpy(Fh).cuda()
    X = torch.full_like(F, float("nan"))
    assert api.poisson_square_solve_noalloc(F, X, 1e-13) == 0
    torch.cuda.synchronize()
    Xo = oracle.poisson_square(Fh, 1e-13)
    err = float(np.abs(X.cpu().numpy() - Xo).max() / np.abs(Xo).max())
    assert err <= TOL_FP64, err


def test_noalloc_rejects_oversize_and_host_buffers(api):
    F = torch.zeros(257, 257, dtype=torch.float64, device="cuda")
    X = torch.zeros_like(F)
    assert api.poisson_square_solve_noalloc(F, X, 1e-13) == -1
    assert "n must be in [1, 256]" in api.lib().fps_last_error().decode()
    Fh = np.zeros((16, 16))
    Xh = np.zeros((16, 16))
    assert api.poisson_square_solve_noalloc(Fh, Xh, 1e-13) == -1
    assert "device memory" in api.lib().fps_last_error().decode()


def test_noalloc_rejects_buffers_of_another_device(api):
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two visible GPUs")
    F = torch.zeros(16, 16, dtype=torch.float64, device="cuda:1")
    X = torch.zeros_like(F)
    with torch.cuda.device(0):
        assert api.lib().fps_poisson_square_solve_noalloc(16, 1e-13, F.data_ptr(), X.data_ptr(), None) == -1
    assert "current device" in api.lib().fps_last_error().decode()
