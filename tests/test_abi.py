"""CPU checks of the C-ABI library: it loads without a GPU, exports every
function declared in include/fps.h, and its host-side mathematics (bands of A~,
Zolotarev shifts, J) agrees with the oracle and with mpmath."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_1710_11259_gb300 import api, build_ext

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build_ext.build()
    return api.lib()


def _declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(fps_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_exports_every_declared_symbol(L):
    declared = _declared_functions()
    assert "fps_plan_create" in declared and "fps_poisson_square_solve" in declared
    for name in declared:
        assert hasattr(L, name), f"{name} declared in include/ but not exported"
    assert set(api.EXPORTED) <= set(declared)


def test_build_arch(L):
    assert L.fps_build_arch() == 103


def test_status_strings(L):
    assert api.status_string(0) == "ok"
    assert api.status_string(-4) == "refinement did not converge"


def test_argument_errors_without_gpu(L):
    """Argument checks run before any CUDA call."""
    with pytest.raises(api.FpsError) as e:
        api.plan_create(0)
    assert e.value.status == -1
    with pytest.raises(api.FpsError) as e:
        api.plan_create(16, tol=1.5)
    assert e.value.status == -1
    with pytest.raises(api.FpsError) as e:
        api.plan_create(16, dim=4)
    assert e.value.status == -1
    with pytest.raises(api.FpsError):
        api.zolotarev_shifts(1.0, 0.0, 2.0, 3.0, 1e-6)


@pytest.mark.parametrize("n", [1, 2, 5, 64, 1001])
def test_square_bands_match_oracle(L, n):
    d, e = api.square_bands(n)
    do, eo = oracle.square_bands(n)
    assert np.abs(d - do).max() <= 1e-15 * np.abs(do).max()
    if n > 2:
        assert np.abs(e - eo).max() <= 1e-15 * np.abs(eo).max()


@pytest.mark.parametrize("n", [1, 16, 64, 512, 2048, 4096, 10000])
@pytest.mark.parametrize("tol", [1e-13, 1e-10, 1e-7])
def test_iteration_count_matches_oracle(L, n, tol):
    a, b, c, d = oracle.square_interval(n)
    p, q = api.zolotarev_shifts(a, b, c, d, tol)
    assert len(q) == oracle.adi_iterations(a, b, c, d, tol)


@pytest.mark.parametrize("case", ["square64", "square4096", "square10000", "fd64", "asym", "cube_outer"])
def test_library_shifts_against_mpmath(L, case):
    """The library's own elliptic-function route to (2.4) against mpmath."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    if case.startswith("square"):
        a, b, c, d = oracle.square_interval(int(case[6:]))
    elif case == "fd64":
        a, b, c, d = -4096.0, -1.0, 1.0, 4096.0
    elif case == "asym":
        a, b, c, d = -1.0, -1e-10, 2e-10, 2.0
    else:
        e2 = (1.0 / (30.0 * 256.0**4)) ** 2
        a, b, c, d = -1.0, -e2, 2 * e2, 2.0
    p, q = api.zolotarev_shifts(a, b, c, d, 1e-13)
    J = len(q)
    A, B, C, D = (mp.mpf(v) for v in (a, b, c, d))
    gam = abs(C - A) * abs(D - B) / (abs(C - B) * abs(D - A))
    alp = -1 + 2 * gam + 2 * mp.sqrt(gam**2 - gam)
    m = 1 - 1 / alp**2
    K = mp.ellipk(m)

    def T(z):
        s = (z + alp) * (-2) / ((z - 1) * (alp - 1))
        return (s * C * (B - A) - A * (B - C)) / (s * (B - A) - (B - C))

    worst = 0.0
    for j in range(J):
        dn = mp.ellipfun("dn", (j + mp.mpf(1) / 2) * K / J, m=m)
        for got, want in ((p[j], T(-alp * dn)), (q[j], T(alp * dn))):
            worst = max(worst, float(abs(got - want) / abs(want)))
    assert worst < 1e-12, worst


def test_library_and_oracle_shifts_agree(L):
    for n in (64, 4096, 10000):
        a, b, c, d = oracle.square_interval(n)
        po, qo = oracle.adi_shifts(a, b, c, d, 1e-13)
        p, q = api.zolotarev_shifts(a, b, c, d, 1e-13)
        assert np.abs(q - qo).max() / 1.0 < 1e-13
        assert (np.abs(q - qo) / qo).max() < 1e-12


@pytest.mark.parametrize("n", [1, 2, 5, 64, 300, 1500])
def test_tight_spectral_interval_contains_spectrum(L, n):
    """Sturm-bisection bounds contain sigma(A~) (eigvalsh) and are tighter than Lemma B.2."""
    lo, hi = api.square_spectral_interval(n, tight=True)
    glo, ghi = api.square_spectral_interval(n, tight=False)
    d, e = oracle.square_bands(n)
    A = np.diag(d)
    for j in range(n - 2):
        A[j, j + 2] = A[j + 2, j] = e[j]
    lam = np.linalg.eigvalsh(A)
    assert lo <= -lam.max() and hi >= -lam.min()
    assert lo >= glo and hi <= ghi
    assert glo == 1.0 / (30.0 * n**4) and ghi == 1.0


def test_legendre_conversion_argument_errors(L):
    """Argument checks of the Legendre conversions run before any CUDA call."""
    import ctypes

    buf = (ctypes.c_double * 64)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    assert L.fps_legendre_to_ctilde(0, p, p, None) == -1           # n < 1
    assert L.fps_legendre_to_ctilde(4, None, p, None) == -1        # NULL
    assert L.fps_legendre_to_ctilde(4, p, p, None) == -1           # overlap
    assert L.fps_solution_to_legendre(0, p, p, None) == -1
    assert L.fps_solution_to_legendre(2, p, None, None) == -1
    assert L.fps_solution_to_legendre(2, p, p, None) == -1         # X inside U
    assert b"overlap" in L.fps_last_error()


def test_binding_rejects_mismatched_buffers():
    """The binding checks shapes before handing raw pointers to the library, so a
    wrong-sized tensor can never make a kernel run past the end of a buffer."""
    plan = api.Plan(0, 8, 2, 1)                      # shape (8, 8); no library call
    with pytest.raises(api.FpsError) as e:
        api._check_plan_buffers(plan, np.zeros((8, 9)), np.zeros((8, 9)))
    assert e.value.status == -1
    with pytest.raises(api.FpsError):
        api._check_plan_buffers(plan, np.zeros((2, 8, 8)), np.zeros((2, 8, 8)))
    with pytest.raises(api.FpsError):
        api._check_plan_buffers(plan, np.zeros((8, 8)), np.zeros((7, 8)))
    api._check_plan_buffers(plan, np.zeros((8, 8)), np.zeros((8, 8)))
    api._check_plan_buffers(plan, np.zeros(64), np.zeros(64))          # packed form
    cube = api.Plan(0, 4, 3, 2)
    api._check_plan_buffers(cube, np.zeros((2, 4, 4, 4)), np.zeros(128))
    with pytest.raises(api.FpsError):
        api._check_plan_buffers(cube, np.zeros((4, 4, 4)), np.zeros(64))
    batch = api.Plan(0, 5, 2, 2, batch_ns=np.array([5, 3]))
    api._check_plan_buffers(batch, np.zeros(2 * 34), np.zeros(2 * 34))
    with pytest.raises(api.FpsError):
        api._check_plan_buffers(batch, np.zeros(2 * 34 - 1), np.zeros(2 * 34))


def test_noalloc_binding_rejects_non_square(L):
    for F, X in [(np.zeros((4, 5)), np.zeros((4, 5))), (np.zeros(16), np.zeros(16)),
                 (np.zeros((4, 4)), np.zeros((5, 5))), (np.zeros((2, 4, 4)), np.zeros((2, 4, 4)))]:
        with pytest.raises(api.FpsError) as e:
            api.poisson_square_solve_noalloc(F, X)
        assert e.value.status == -1


def test_dirichlet_argument_errors(L):
    """The Dirichlet entry points reject a NULL plan before any CUDA call, and the
    binding rejects buffers of the wrong shape and batched or cube plans."""
    import ctypes

    buf = (ctypes.c_double * 64)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    assert L.fps_poisson_dirichlet_solve(None, p, p, p) == -1
    assert L.fps_poisson_dirichlet_adjoint(None, p, p, p) == -1
    plan = api.Plan(0, 8, 2, 1)
    G, bc, U = np.zeros((8, 8)), np.zeros((4, 10)), np.zeros((10, 10))
    for args in [(np.zeros((8, 9)), bc, U), (G, np.zeros((4, 9)), U), (G, bc, np.zeros((8, 8))),
                 (G, np.zeros((3, 10)), U)]:
        with pytest.raises(api.FpsError) as e:
            api.poisson_dirichlet_solve(plan, *args)
        assert e.value.status == -1 and "shape" in str(e.value)
    with pytest.raises(api.FpsError):
        api.poisson_dirichlet_adjoint(plan, np.zeros((8, 8)), G, bc)
    two = api.Plan(0, 8, 2, 2)
    with pytest.raises(api.FpsError):
        api.poisson_dirichlet_solve(two, G, bc, U)              # nrhs = 2 needs a leading axis
    for other in [api.Plan(0, 8, 3, 1), api.Plan(0, 8, 2, 1, batch_ns=np.array([8, 4]))]:
        with pytest.raises(api.FpsError) as e:
            api.poisson_dirichlet_solve(other, G, bc, U)
        assert "single square or rectangle" in str(e.value)
