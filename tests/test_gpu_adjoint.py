"""GPU checks of the adjoint (torch.autograd through fps_poisson_adjoint).

Pins: self-adjointness of the GPU solve map, the dense adjoint (M (x) D + D (x) M)^{-T}
at small n, torch.autograd.gradcheck, and central finite differences of
L = 0.5 ||X - U*||_F^2 along 16 seeded unit directions at n = 10^4 (FP32 sweeps +
FP64 refinement), relative error <= 1e-6.  L is quadratic in F, so central
differences carry no truncation error for any step; L itself is dominated by the
constant 0.5 ||U*||^2 and the refined solve is linear only to its tolerance, so the
step is taken large (h ||V|| = 10 ||F||) to lift the difference above that noise."""
import numpy as np
import pytest

import oracle
from paper_1710_11259_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_11259_gb300 import api, autograd, build_ext

    build_ext.build()
    api.lib()
    return api, autograd


@pytest.mark.parametrize("n", [50, 300])
def test_gpu_solve_map_is_self_adjoint(mods, n):
    """<P a, b> = <a, P b> for white-noise a, b, up to rounding measured against the
    size of the summands (Cauchy-Schwarz scale ||P a|| ||b||): the inner products
    cancel heavily (|<P a, b>| = 0.16 at n = 50), so a bound relative to the sum
    itself would measure the cancellation.  n = 50 runs the one-launch small-n path,
    n = 300 the pass kernels."""
    api, _ = mods
    a = torch.from_numpy(inputs.gaussian(31, (n, n))).cuda()
    b = torch.from_numpy(inputs.gaussian(32, (n, n))).cuda()
    plan = api.plan_create(n, 2, 1e-13, "fp64")
    Pa = api.poisson_square_solve(plan, a)
    Pb = api.poisson_square_solve(plan, b)
    lhs, rhs = float((Pa * b).sum()), float((a * Pb).sum())
    scale = max(float(Pa.norm() * b.norm()), float(a.norm() * Pb.norm()))
    api.plan_destroy(plan)
    assert abs(lhs - rhs) <= 1e-13 * scale, (lhs, rhs, scale)


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_adjoint_matches_dense_transpose(mods, precision):
    api, autograd = mods
    n = 16
    d, e = oracle.M_bands(n)
    M = np.diag(d)
    for j in range(n - 2):
        M[j, j + 2] = M[j + 2, j] = e[j]
    Dm = np.diag([-(j * (j + 3) + 2.0) for j in range(n)])
    L = np.kron(M, Dm) + np.kron(Dm, M)
    G = inputs.gaussian(33, (n, n))
    want = np.linalg.solve(L.T, G.ravel()).reshape(n, n)     # dL/dF for dL/dX = G
    plan = api.plan_create(n, 2, 1e-13 if precision == "fp64" else 1e-12, precision)
    F = torch.from_numpy(inputs.square_rhs(n, 34)).cuda().requires_grad_(True)
    X = autograd.poisson_square(F, plan)
    X.backward(torch.from_numpy(G).cuda())
    got = F.grad.cpu().numpy()
    api.plan_destroy(plan)
    assert np.abs(got - want).max() / np.abs(want).max() <= (1e-12 if precision == "fp64" else 1e-10)


def test_gradcheck_small(mods):
    api, autograd = mods
    n = 6
    plan = api.plan_create(n, 2, 1e-13, "fp64")
    F = torch.from_numpy(inputs.square_rhs(n, 35)).cuda().requires_grad_(True)
    ok = torch.autograd.gradcheck(lambda f: autograd.poisson_square(f, plan), (F,), eps=1e-6, atol=1e-8)
    api.plan_destroy(plan)
    assert ok


@pytest.mark.parametrize("n,precision,tol", [(300, "fp64", 1e-13), (300, "fp32_refine", 1e-10),
                                             (10000, "fp64", 1e-13)])
def test_adjoint_against_central_differences(mods, n, precision, tol):
    """Config of the n = 10^4 workload: F = g/((1+j)(1+k)) seed 3, U* seed 4, 16 FD directions (seed 7).

    L is exactly quadratic in F, so the central difference carries no truncation
    error; with h ||V|| = 10 ||F|| its FP64 rounding stays near 1e-7 at n = 10^4.  The
    FP32-refined solve is linear only to its accuracy, which this quotient amplifies
    to ~1e-6 at n = 10^4 whatever the stopping tolerance (measured 1.6e-6 at 1e-10
    and 1.05e-6 at 1e-12), so its n = 10^4 gradient is checked against the FP64
    gradient instead (next test)."""
    api, autograd = mods
    F0 = torch.from_numpy(inputs.square_rhs(n, 3, power=1)).cuda()
    Ustar = torch.from_numpy(inputs.gaussian(4, (n, n))).cuda()
    V = inputs.unit_directions(7, 16, (n, n))
    plan = api.plan_create(n, 2, tol, precision)

    def loss(F):
        X = autograd.poisson_square(F, plan)
        return 0.5 * ((X - Ustar) ** 2).sum()

    F = F0.clone().requires_grad_(True)
    loss(F).backward()
    g = F.grad
    h = 10.0 * float(F0.norm())
    gnorm = float(g.norm())
    worst = 0.0
    with torch.no_grad():
        for k in range(V.shape[0]):
            Vk = torch.from_numpy(V[k]).cuda()
            fd = (float(loss(F0 + h * Vk)) - float(loss(F0 - h * Vk))) / (2 * h)
            an = float((g * Vk).sum())
            # relative to the directional derivative; directions almost orthogonal to
            # the gradient are measured against 1e-3 ||dL/dF|| instead
            worst = max(worst, abs(fd - an) / max(abs(an), 1e-3 * gnorm))
    api.plan_destroy(plan)
    assert worst <= 1e-6, worst


def test_refined_gradient_matches_fp64_gradient_n10000(mods):
    """dL/dF through the FP32-refined solve (tol 1e-10) against dL/dF through the FP64
    solve at n = 10^4, element by element: both are the adjoint solve of X - U*.  The
    refinement bounds its residual relative to the largest coefficient of the right-
    hand side; X - U* is white noise (no decay), and the measured difference is
    1.4e-10 of max |dL/dF|, so the bar is 1e-9 (the workload's bar for gradients is
    1e-6 against finite differences)."""
    api, autograd = mods
    n = 10000
    F0 = torch.from_numpy(inputs.square_rhs(n, 3, power=1)).cuda()
    Ustar = torch.from_numpy(inputs.gaussian(4, (n, n))).cuda()
    grads = {}
    for precision, tol in (("fp64", 1e-13), ("fp32_refine", 1e-10)):
        plan = api.plan_create(n, 2, tol, precision)
        F = F0.clone().requires_grad_(True)
        X = autograd.poisson_square(F, plan)
        (0.5 * ((X - Ustar) ** 2).sum()).backward()
        grads[precision] = F.grad.detach()
        api.plan_destroy(plan)
        del X, F
    err = float((grads["fp32_refine"] - grads["fp64"]).abs().max() / grads["fp64"].abs().max())
    assert err <= 1e-9, err
