"""The library's Chebyshev coefficients (bt_alpha_chebyshev, host code) against
the oracle's, and its exact admissibility check of alpha (q > 0 on [0, 1],
by a Sturm sequence; bt_params_check, host code) against hand-factored
polynomials.  No GPU needed."""
import ctypes

import numpy as np
import pytest

from oracle import bt_oracle as orc
from paper_2503_15269_gb300 import binding as bb


@pytest.fixture(scope="module")
def built():
    from paper_2503_15269_gb300 import build
    build.build()
    return bb.lib()


@pytest.mark.parametrize("m", range(1, 9))
@pytest.mark.parametrize("rho", [0.3, 0.9, 0.985, 0.999])
def test_library_matches_oracle(built, m, rho):
    st, a = bb.bt_alpha_chebyshev(m, rho)
    assert st == bb.BT_OK
    assert np.allclose(a, orc.chebyshev_alpha(m, rho), rtol=1e-9, atol=1e-12)


def test_bad_arguments(built):
    for m, rho in [(0, 0.5), (9, 0.5), (2, 0.0), (2, 1.0), (2, float("nan"))]:
        assert bb.bt_alpha_chebyshev(m, rho)[0] == bb.BT_ERR_ARG


def _params(alpha, a=1.0):
    """bt_params on the host only (make_params would ask torch for a stream)."""
    q = bb.bt_params()
    bb.lib().bt_params_init(ctypes.byref(q))
    q.m = len(alpha)
    q.a = a
    arr = (ctypes.c_double * len(alpha))(*alpha)
    q.alpha = ctypes.cast(arr, ctypes.POINTER(ctypes.c_double))
    return q, arr


# (alpha, admissible): q(h) = sum alpha_j h^j factored by hand
CASES = [
    ([1.0, -3.0, 2.0], False),        # (1 - h)(1 - 2h): zero at 1/2 and 1
    ([1.0, -2.9, 2.0], False),        # roots 0.565, 0.885 inside (0, 1)
    ([1.0, -2.0, 1.0], False),        # (1 - h)^2: double root at 1
    ([1.0, -3.5, 2.5], False),        # (1 - h)(1 - 2.5 h): roots 0.4 and 1
    ([1.0, -2.5, 2.0], True),         # no real root (discriminant < 0)
    ([1.0, 1.5, -1.0], True),         # roots -0.5 and 2, outside [0, 1]
    ([1.0, -1.0], False),             # 1 - h: zero at 1
    ([1.0, -0.99], True),             # root 1.0101 > 1
    ([1.0, 7.0], True),               # PolyCoeff m = 2
    ([1.0, 0.0, 0.0, -1.2], False),   # 1 - 1.2 h^3: root 0.941
]


@pytest.mark.parametrize("alpha,ok", CASES)
def test_admissibility_is_exact(built, alpha, ok):
    h = np.linspace(0.0, 1.0, 200001)
    assert (np.polynomial.polynomial.polyval(h, alpha).min() > 0) == ok  # the hand factoring
    q, keep = _params(alpha)
    assert bb.lib().bt_params_check(ctypes.byref(q)) == (bb.BT_OK if ok else bb.BT_ERR_PARAM)


@pytest.mark.parametrize("m", [2, 3, 4, 6, 8])
def test_chebyshev_coefficients_are_admissible(built, m):
    st, a = bb.bt_alpha_chebyshev(m, 0.985)
    q, keep = _params(a)
    assert bb.lib().bt_params_check(ctypes.byref(q)) == bb.BT_OK
    q, keep = _params(a, a=0.5)   # coefficients other than ones need a = 1
    assert bb.lib().bt_params_check(ctypes.byref(q)) == bb.BT_ERR_PARAM
