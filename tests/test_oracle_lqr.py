"""Pins of the oracle's LQR Schur-complement formation and dual-to-primal
recovery (the reading of Sec. 5's construction: the equality-constrained QP
of an LQR problem, its KKT system, and the Schur complement w.r.t. the
Hessian).  Each test checks the oracle against something other than itself:
the bordered KKT system solved as one dense system, the closed form of the
Schur blocks, hand-derived scalars, and the QP's optimality."""
import numpy as np
import pytest

from oracle import bt_oracle as orc
from paper_2503_15269_gb300 import workloads as wl


def _args(d):
    return d.A, d.Bm, d.Q, d.R, d.q, d.r, d.c


@pytest.mark.parametrize("N,n,m", [(1, 3, 2), (2, 2, 1), (5, 4, 2), (9, 6, 3), (12, 5, 5)])
def test_schur_and_recovery_solve_the_kkt_system(N, n, m):
    """[G C^T; C 0][z; lam] = [-g; c] solved as one dense system: its lam
    solves S lam = gamma and its z is the recovery of lam."""
    d = wl.small_lqr(1, N, n, m)
    G, g, C, c = orc.lqr_dense(*_args(d))
    nz, nl = G.shape[0], C.shape[0]
    K = np.block([[G, C.T], [C, np.zeros((nl, nl))]])
    sol = np.linalg.solve(K, np.concatenate([-g, c]))
    z, lam = sol[:nz], sol[nz:].reshape(N, n)
    D, O, gamma = orc.lqr_schur(*_args(d))
    S = orc.assemble(D, O)
    assert np.allclose(S @ lam.reshape(-1), gamma.reshape(-1), rtol=1e-10, atol=1e-10)
    assert np.allclose(orc.direct_solve(D, O, gamma), lam, rtol=1e-9, atol=1e-10)
    x, u = orc.lqr_recover(d.A, d.Bm, d.Q, d.R, d.q, d.r, lam)
    zz = np.concatenate([np.concatenate([x[k], u[k]]) if k < N - 1 else x[k] for k in range(N)])
    assert np.allclose(zz, z, rtol=1e-10, atol=1e-10)


def test_schur_blocks_match_closed_form():
    """Diagonal Q, R: the blocks equal the closed form of the ocp generator
    (D_0 = Q_0^-1, D_{k+1} = A_k Q_k^-1 A_k^T + B_k R_k^-1 B_k^T + Q_{k+1}^-1,
    O_k = -Q_k^-1 A_k^T), drawn from the same seed."""
    N, n, m = 6, 4, 2
    rng = np.random.Generator(np.random.PCG64(77))
    inst = wl.ocp_instance(rng, N, n, m)
    rng = np.random.Generator(np.random.PCG64(77))
    A = np.eye(n) + 0.05 * rng.standard_normal((N - 1, n, n))
    Bm = 0.05 * rng.standard_normal((N - 1, n, m))
    Q = np.stack([np.diag(v) for v in rng.uniform(1.0, 10.0, (N, n))])
    R = np.stack([np.diag(v) for v in rng.uniform(0.1, 1.0, (N - 1, m))])
    D, O, gamma = orc.lqr_schur(A, Bm, Q, R, np.zeros((N, n)), np.zeros((N - 1, m)), np.zeros((N, n)))
    assert np.allclose(D, inst.D, rtol=1e-12, atol=1e-14)
    assert np.allclose(O, inst.O, rtol=1e-12, atol=1e-14)
    assert np.abs(gamma).max() == 0.0


def test_scalar_case_by_hand():
    """N = 2, n = m = 1: S = [[1/Q0, -A/Q0], [-A/Q0, A^2/Q0 + B^2/R + 1/Q1]],
    gamma_0 = -(c0 + q0/Q0), gamma_1 = -(c1 + q1/Q1 - A q0/Q0 - B r/R)."""
    a, b, Q0, Q1, R0, q0, q1, r0, c0, c1 = 1.3, 0.7, 2.0, 5.0, 0.5, 0.3, -1.1, 0.9, 0.4, -0.2
    D, O, gamma = orc.lqr_schur(np.array([[[a]]]), np.array([[[b]]]), np.array([[[Q0]], [[Q1]]]),
                                np.array([[[R0]]]), np.array([[q0], [q1]]), np.array([[r0]]),
                                np.array([[c0], [c1]]))
    assert np.isclose(D[0, 0, 0], 1 / Q0) and np.isclose(D[1, 0, 0], a * a / Q0 + b * b / R0 + 1 / Q1)
    assert np.isclose(O[0, 0, 0], -a / Q0)
    assert np.isclose(gamma[0, 0], -(c0 + q0 / Q0))
    assert np.isclose(gamma[1, 0], -(c1 + q1 / Q1 - a * q0 / Q0 - b * r0 / R0))
    lam = np.array([[0.25], [-0.5]])
    x, u = orc.lqr_recover(np.array([[[a]]]), np.array([[[b]]]), np.array([[[Q0]], [[Q1]]]),
                           np.array([[[R0]]]), np.array([[q0], [q1]]), np.array([[r0]]), lam)
    # z = -G^-1 (g + C^T lam): x0 = -(q0 + lam0 - a lam1)/Q0, u0 = -(r0 - b lam1)/R0, x1 = -(q1 + lam1)/Q1
    assert np.isclose(x[0, 0], -(q0 + 0.25 + a * 0.5) / Q0)
    assert np.isclose(u[0, 0], -(r0 + b * 0.5) / R0)
    assert np.isclose(x[1, 0], -(q1 - 0.5) / Q1)


def test_recovered_z_is_the_qp_minimiser():
    """The z from S lam = gamma is feasible (C z = c) and no feasible step
    (a null-space direction of C) lowers the objective."""
    N, n, m = 7, 3, 2
    d = wl.small_lqr(2, N, n, m)
    D, O, gamma = orc.lqr_schur(*_args(d))
    lam = orc.direct_solve(D, O, gamma)
    x, u = orc.lqr_recover(d.A, d.Bm, d.Q, d.R, d.q, d.r, lam)
    z = np.concatenate([np.concatenate([x[k], u[k]]) if k < N - 1 else x[k] for k in range(N)])
    G, g, C, c = orc.lqr_dense(*_args(d))
    assert np.allclose(C @ z, c, atol=1e-10)
    f = lambda v: 0.5 * v @ G @ v + g @ v
    null = np.linalg.svd(C)[2][C.shape[0]:].T
    rng = np.random.default_rng(0)
    for _ in range(20):
        step = null @ rng.standard_normal(null.shape[1]) * 1e-3
        assert f(z + step) > f(z)
