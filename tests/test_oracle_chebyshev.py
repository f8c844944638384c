"""Pins of the oracle's Chebyshev polynomial coefficients (the choice of
alpha beyond grid search): a hand-derived closed form, the minimax
equioscillation of the preconditioned spectrum, optimality against other
coefficients, positivity of q on [0, 1], and the iteration counts it buys."""
import numpy as np
import pytest

from oracle import bt_oracle as orc
from paper_2503_15269_gb300 import workloads as wl


def phi(alpha, h):
    return np.polynomial.polynomial.polyval(h, alpha) * (1.0 - h)


def test_m1_is_the_plain_preconditioner():
    assert np.array_equal(orc.chebyshev_alpha(1, 0.9), [1.0])


@pytest.mark.parametrize("rho", [0.5, 0.9, 0.98197, 0.999])
def test_m2_closed_form(rho):
    """By hand: T_2(x) = 2x^2 - 1 at x = 2h/rho - 1 gives
    1 - p(h) = (1 - h)(A + B h) / T_2(2/rho - 1), A = 8/rho^2 - 8/rho,
    B = 8/rho^2, so alpha = (1, B/A) = (1, 1/(1 - rho))."""
    a = orc.chebyshev_alpha(2, rho)
    assert np.allclose(a, [1.0, 1.0 / (1.0 - rho)], rtol=1e-12)


@pytest.mark.parametrize("m", [2, 3, 4, 5])
@pytest.mark.parametrize("rho", [0.7, 0.95, 0.985])
def test_equioscillation(m, rho):
    """c phi(h) = 1 - p(h) stays within 1 +- eps on [0, rho], eps =
    1 / T_m((2 - rho)/rho) = 1 / cosh(m arccosh((2 - rho)/rho)), and touches
    both ends m + 1 times."""
    a = orc.chebyshev_alpha(m, rho)
    h = np.linspace(0.0, rho, 20001)
    f = phi(a, h)
    eps = 1.0 / np.cosh(m * np.arccosh((2.0 - rho) / rho))
    c = 1.0 / (0.5 * (f.max() + f.min()))
    g = c * f
    assert np.isclose(g.max(), 1 + eps, rtol=1e-6) and np.isclose(g.min(), 1 - eps, rtol=1e-6)
    ext = np.cos(np.pi * np.arange(m + 1) / m)              # extrema of T_m
    he = rho * (ext + 1.0) / 2.0
    assert np.allclose(np.abs(c * phi(a, he) - 1.0), eps, rtol=1e-6)


@pytest.mark.parametrize("m", [2, 3, 4])
def test_no_other_alpha_does_better(m):
    rho = 0.95
    h = np.linspace(0.0, rho, 4001)
    f = phi(orc.chebyshev_alpha(m, rho), h)
    best = f.max() / f.min()
    rng = np.random.default_rng(m)
    a0 = orc.chebyshev_alpha(m, rho)
    for _ in range(200):
        a = a0 * (1 + 0.05 * rng.standard_normal(m))
        a[0] = 1.0
        g = phi(a, h)
        if g.min() > 0:
            assert g.max() / g.min() >= best * (1 - 1e-9)


@pytest.mark.parametrize("m", [2, 3, 4, 6])
def test_q_positive_on_unit_interval(m):
    """q > 0 on [0, 1] (so M^-1 stays SPD for every spectrum of H_opt in
    [0, 1)), although the coefficients alternate in sign."""
    a = orc.chebyshev_alpha(m, 0.985)
    h = np.linspace(0.0, 1.0, 100001)
    assert np.polynomial.polynomial.polyval(h, a).min() > 0


def test_fewer_iterations_than_polycoeff_at_m3_m4():
    """On the LQR family (rho(H_opt) ~ 0.98): Chebyshev coefficients at
    m = 3, 4 need fewer PCG iterations than PolyCoeff's alpha_{m-1} = 7."""
    inst = wl.small_ocp(400, 128, 12)
    for m in (3, 4):
        pc = orc.pcg_opt(inst.D, inst.O, inst.b, [1.0] * (m - 1) + [7.0], 1e-8, 3000).iters
        ch = orc.pcg_opt(inst.D, inst.O, inst.b, orc.chebyshev_alpha(m, 0.985), 1e-8, 3000).iters
        assert ch < pc, (m, ch, pc)


def test_power_rho_approaches_the_dense_spectral_radius():
    """The power-iteration estimate against the eigenvalues of the dense
    H_opt (from apply_H_opt on the columns of I): the error shrinks with the
    step count.  H_opt is not symmetric, so ||H v|| / ||v|| is not bounded by
    rho and may end slightly above it."""
    inst = wl.small_ocp(500, 16, 6)
    B = orc.opt_blocks(inst.D, inst.O)
    N, n = 16, 6
    eye = np.eye(N * n)
    H = np.column_stack([orc.apply_H_opt(B, eye[:, k].reshape(N, n)).reshape(-1) for k in range(N * n)])
    rho = np.abs(np.linalg.eigvals(H)).max()
    est = [orc.power_rho(inst.D, inst.O, k) for k in (50, 400)]
    assert abs(rho - est[1]) < abs(rho - est[0])
    assert abs(rho - est[1]) < 1e-4


def test_ritz_rho_converges_faster_than_power_iteration():
    """Ritz values from 60 PCG iterations against the dense spectral radius:
    closer than 400 power-iteration steps (1e-15 vs 5e-6 on this case)."""
    inst = wl.small_ocp(500, 16, 6)
    B = orc.opt_blocks(inst.D, inst.O)
    N, n = 16, 6
    eye = np.eye(N * n)
    H = np.column_stack([orc.apply_H_opt(B, eye[:, k].reshape(N, n)).reshape(-1) for k in range(N * n)])
    rho = np.abs(np.linalg.eigvals(H)).max()
    b = np.random.default_rng(3).standard_normal((N, n))
    est = orc.ritz_rho(inst.D, inst.O, b, 60)
    assert abs(est - rho) < 1e-8
    assert abs(orc.ritz_rho(inst.D, inst.O, b, 40) - rho) < abs(orc.ritz_rho(inst.D, inst.O, b, 20) - rho)
    assert abs(est - rho) < abs(orc.power_rho(inst.D, inst.O, 400) - rho)
