"""Host side of the cylinder modes (Sec. 4.1, Case 1), no GPU: the library's closed
forms of L1 and Q against the oracle's quadrature matrices, and the library's
power-iteration interval of sigma(A_k) against the oracle's dense eigenvalues."""
import numpy as np
import pytest

from oracle import cylinder as cyl
from paper_1710_11259_gb300 import api


@pytest.fixture(scope="module")
def L():
    from paper_1710_11259_gb300 import build_ext

    build_ext.build()
    return api.lib()


@pytest.mark.parametrize("n", [4, 7, 20, 33])
def test_operators_match_oracle(L, n):
    L1, Q = api.cylinder_operators(n)
    P0, Qo, M, D = cyl.mode_operators(n, 0)
    assert np.abs(L1 - P0).max() <= 1e-11 * np.abs(P0).max()
    assert np.abs(Q - Qo).max() <= 1e-13


@pytest.mark.parametrize("n,k", [(8, 2), (24, 2), (24, 3), (32, 7), (48, 24), (64, 2)])
def test_mode_interval_contains_spectrum(L, n, k):
    a, b = api.cylinder_mode_interval(n, k)
    P, Q, M, D = cyl.mode_operators(n, k)
    ev = np.linalg.eigvals(np.linalg.solve(P, Q))
    assert np.abs(ev.imag).max() <= 1e-10 * np.abs(ev).max()
    ev = ev.real
    assert a <= ev.min() and ev.max() <= b < 0
    assert a >= 1.1 * ev.min() and b <= 0.9 * ev.max()   # not much wider than the spectrum


def test_cylinder_argument_errors(L):
    import ctypes

    h = ctypes.c_void_p()
    assert L.fps_plan_create_cylinder(ctypes.byref(h), 3, 2, 4, 1e-10, 1, None) == -1    # n < 4
    assert L.fps_plan_create_cylinder(ctypes.byref(h), 16, 1, 4, 1e-10, 1, None) == -1   # kmin < 2
    assert L.fps_plan_create_cylinder(ctypes.byref(h), 16, 5, 4, 1e-10, 1, None) == -1   # kmax < kmin
    assert L.fps_plan_create_cylinder(ctypes.byref(h), 16, 2, 4, 1.5, 1, None) == -1     # tol
    assert L.fps_poisson_cylinder_solve(None, None, None) == -1
    with pytest.raises(api.FpsError):
        api.cylinder_mode_interval(16, 1)
    with pytest.raises(api.FpsError):
        api.cylinder_mode_interval(4097, 2)
    with pytest.raises(api.FpsError):
        api.cylinder_operators(4097)
