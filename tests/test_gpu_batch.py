"""GPU parity of the batched solve (many squares of different n, several
right-hand sides each, FP32 sweeps + FP64 refinement), through the C ABI.

Every (problem, right-hand side) is compared with the CPU oracle to the FP32+refine
bar, relative max-coefficient error <= 1e-10; at the full workload (512 problems,
n log-uniform in [32, 2048], 4 RHS) a sample of problems is compared with the
oracle and every right-hand side must meet the residual target."""
import numpy as np
import pytest

import oracle
from paper_1710_11259_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_REFINE = 1e-10


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_11259_gb300 import api as _api
    from paper_1710_11259_gb300 import build_ext

    build_ext.build()
    _api.lib()
    return _api


def _pack(rhs):
    return np.concatenate([r.ravel() for r in rhs])


def _unpack(x, ns, nrhs):
    out, o = [], 0
    for n in ns:
        sz = nrhs * n * n
        out.append(x[o:o + sz].reshape(nrhs, n, n))
        o += sz
    return out


def _relmax(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("nrhs", [1, 2])
def test_small_batch_matches_oracle(api, nrhs):
    ns = [1, 2, 3, 5, 33, 64, 100, 257, 64]
    rng = np.random.default_rng(40 + nrhs)
    rhs = []
    for n in ns:
        w = inputs.decay_weights(n, 2)
        rhs.append(rng.standard_normal((nrhs, n, n)) * w[None, :, None] * w[None, None, :])
    F = torch.from_numpy(_pack(rhs)).cuda()
    plan = api.plan_create_batched(ns, nrhs=nrhs, tol=1e-10, precision="fp32_refine")
    X = api.poisson_square_solve(plan, F)
    torch.cuda.synchronize()
    info = api.plan_info(plan)
    api.plan_destroy(plan)
    assert info["batch"] == len(ns) and info["last_residual"] <= 1e-10
    Xs = _unpack(X.cpu().numpy(), ns, nrhs)
    for p, n in enumerate(ns):
        for r in range(nrhs):
            Xo = oracle.poisson_square(rhs[p][r], 1e-13)
            assert _relmax(Xs[p][r], Xo) <= TOL_REFINE, (n, r)


def test_batch_with_zero_rhs_and_host_pointers(api):
    ns = [40, 17]
    F = np.concatenate([inputs.square_rhs(40, 1).ravel(), np.zeros(17 * 17)])
    plan = api.plan_create_batched(ns, nrhs=1, tol=1e-10, precision="fp32_refine")
    X = api.poisson_square_solve(plan, F)   # numpy in/out: staged by the library
    api.plan_destroy(plan)
    assert np.all(X[40 * 40:] == 0.0)
    assert _relmax(X[:1600].reshape(40, 40), oracle.poisson_square(F[:1600].reshape(40, 40), 1e-13)) <= TOL_REFINE


def test_batched_workload_512_problems(api):
    """512 squares, n = round(exp(U(ln 32, ln 2048))) seed 5, 4 RHS each, F = g/((1+j)^2(1+k)^2)."""
    ns, rhs = inputs.batch_problems(seed=5)
    ns = [int(n) for n in ns]
    F = torch.from_numpy(_pack(rhs)).cuda()
    plan = api.plan_create_batched(ns, nrhs=4, tol=1e-10, precision="fp32_refine")
    X = api.poisson_square_solve(plan, F)
    torch.cuda.synchronize()
    info = api.plan_info(plan)
    api.plan_destroy(plan)
    assert info["batch"] == 512 and info["last_residual"] <= 1e-10
    Xs = _unpack(X.cpu().numpy(), ns, 4)
    del X, F
    # every one of the 2048 (problem, right-hand side) pairs, element by element
    worst = 0.0
    for p in range(len(ns)):
        for r in range(4):
            e = _relmax(Xs[p][r], oracle.poisson_square(rhs[p][r], 1e-13))
            worst = max(worst, e)
            assert e <= TOL_REFINE, (p, ns[p], r, e)
    assert worst <= TOL_REFINE


def test_autotuner_picks_and_caches(api, tmp_path, monkeypatch):
    """The segment length is picked by timing complete candidate engines on the plan's
    sizes, then cached per GPU and size list; the tuned plan still matches the oracle."""
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("FPS_AUTOTUNE_CACHE", str(cache))
    monkeypatch.delenv("FPS_AUTOTUNE", raising=False)
    ns = [300, 257, 64, 33]
    plan = api.plan_create_batched(ns, nrhs=2, tol=1e-10, precision="fp32_refine")
    chosen = api.plan_info(plan)["seg_len"]
    chosen_chain = api.plan_info(plan)["chain_mode"]
    api.plan_destroy(plan)
    assert chosen in {64, 128} and chosen_chain in {1, 2}
    assert cache.read_text().split()[1:3] == [str(chosen), str(chosen_chain)]
    lines = cache.read_text().split("\n")
    assert len([ln for ln in lines if ln.strip()]) == 1
    plan = api.plan_create_batched(ns, nrhs=2, tol=1e-10, precision="fp32_refine")
    assert api.plan_info(plan)["seg_len"] == chosen and api.plan_info(plan)["chain_mode"] == chosen_chain
    F = torch.from_numpy(np.concatenate([inputs.square_rhs(n, 60 + n).ravel() for n in ns for _ in range(2)])).cuda()
    X = api.poisson_square_solve(plan, F)
    torch.cuda.synchronize()
    api.plan_destroy(plan)
    assert len([ln for ln in cache.read_text().split("\n") if ln.strip()]) == 1
    x = X.cpu().numpy()
    f = F.cpu().numpy()
    o = 0
    for n in ns:
        for _ in range(2):
            Xo = oracle.poisson_square(f[o:o + n * n].reshape(n, n), 1e-13)
            assert _relmax(x[o:o + n * n].reshape(n, n), Xo) <= TOL_REFINE
            o += n * n


@pytest.mark.parametrize("seg,chain", [("64", 1), ("64", 2), ("128", 1), ("128", 2)])
def test_both_segment_lengths_match_oracle(api, tmp_path, monkeypatch, seg, chain):
    """Each compiled segment length and chain-kernel load batching, forced through the
    cache, on sizes with a short last segment (n = 200, 321) and a single segment (n = 33)."""
    ns = [321, 200, 33]
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("FPS_AUTOTUNE_CACHE", str(cache))
    monkeypatch.delenv("FPS_AUTOTUNE", raising=False)
    plan = api.plan_create_batched(ns, nrhs=1, tol=1e-10, precision="fp32_refine")
    key = cache.read_text().split()[0]
    api.plan_destroy(plan)
    cache.write_text(f"{key} {seg} {chain}\n")
    plan = api.plan_create_batched(ns, nrhs=1, tol=1e-10, precision="fp32_refine")
    assert api.plan_info(plan)["seg_len"] == int(seg) and api.plan_info(plan)["chain_mode"] == chain
    rng = np.random.default_rng(77)
    rhs = [rng.standard_normal((1, n, n)) * inputs.decay_weights(n, 2)[None, :, None] *
           inputs.decay_weights(n, 2)[None, None, :] for n in ns]
    X = api.poisson_square_solve(plan, torch.from_numpy(_pack(rhs)).cuda())
    torch.cuda.synchronize()
    api.plan_destroy(plan)
    Xs = _unpack(X.cpu().numpy(), ns, 1)
    for p, n in enumerate(ns):
        assert _relmax(Xs[p][0], oracle.poisson_square(rhs[p][0], 1e-13)) <= TOL_REFINE, n
