"""Failure paths of the square solve, driven from the host (no GPU fault is made):
the refinement that misses its target (FPS_ERR_NOT_CONVERGED, last iterate kept in X)
and a corrupted shift list rejected before any kernel runs."""
import numpy as np
import pytest

import oracle
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


def test_refinement_capped_reports_not_converged(api, monkeypatch):
    """One refinement round cannot reach 1e-13: the solve returns NOT_CONVERGED and X
    holds that round's iterate (the FP32 inner solve's accuracy, ~1e-7)."""
    monkeypatch.setenv("FPS_MAX_REFINE_ROUNDS", "1")
    monkeypatch.setenv("FPS_AUTOTUNE", "0")
    n = 300
    F = inputs.square_rhs(n, 21)
    plan = api.plan_create(n, 2, 1e-13, "fp32_refine")
    Fd = torch.from_numpy(F).cuda()
    X = torch.full_like(Fd, float("nan"))
    with pytest.raises(api.FpsError) as e:
        api.poisson_square_solve(plan, Fd, X)
    assert e.value.status == -4
    info = api.plan_info(plan)
    api.plan_destroy(plan)
    assert info["refine_rounds"] == 1 and info["last_residual"] > 1e-13
    Xo = oracle.poisson_square(F, 1e-13)
    err = float(np.abs(X.cpu().numpy() - Xo).max() / np.abs(Xo).max())
    assert np.isfinite(X.cpu().numpy()).all() and err < 1e-4, err


@pytest.mark.parametrize("fault", ["nan", "neg"])
@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_corrupted_shift_list_rejected_at_plan_creation(api, monkeypatch, fault, precision):
    monkeypatch.setenv("FPS_INJECT_SHIFT_FAULT", fault)
    monkeypatch.setenv("FPS_AUTOTUNE", "0")
    with pytest.raises(api.FpsError) as e:
        api.plan_create(64, 2, 1e-10, precision)
    assert e.value.status == -1 and "shift list" in str(e.value)
    monkeypatch.delenv("FPS_INJECT_SHIFT_FAULT")
    plan = api.plan_create(64, 2, 1e-10, precision)   # the same request without the fault
    api.plan_destroy(plan)
