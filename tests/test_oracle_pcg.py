"""Pins for the oracle's PCG: agreement with the direct solve within the
kappa * tol bound, the exact-arithmetic iteration bound d_Nna on tiny cases,
the footnote's Jacobi equivalence and the status paths."""
import numpy as np
import pytest

from oracle import bt_oracle as orc
from paper_2503_15269_gb300 import workloads as wl


@pytest.mark.parametrize("alpha", [(1.0,), (1.0, 1.0), (1.0, 7.0)])
def test_pcg_config0_matches_direct(alpha):
    inst = wl.config0()
    res = orc.pcg_opt(inst.D, inst.O, inst.b, alpha, 1e-10, 500)
    assert res.status == orc.OK
    x = orc.direct_solve(inst.D, inst.O, inst.b)
    S = orc.assemble(inst.D, inst.O)
    kappa = np.linalg.cond(S)
    assert np.linalg.norm(res.x - x) / np.linalg.norm(x) <= kappa * 1e-10
    assert np.linalg.norm(orc.spmv(inst.D, inst.O, res.x) - inst.b) <= 1e-10 * np.linalg.norm(inst.b) * 1.0001


@pytest.mark.parametrize("N,n", [(4, 2), (5, 2), (6, 1), (7, 2)])
@pytest.mark.parametrize("m", [1, 2])
def test_pcg_iterations_bounded_by_distinct_eigenvalues(N, n, m):
    """In exact arithmetic CG ends in at most d_Nna steps (Sec. 4.3); at these
    tiny well-conditioned sizes FP64 follows it to within one step."""
    inst = wl.small_ocp(20, N, n)
    res = orc.pcg_opt(inst.D, inst.O, inst.b, [1.0] * m, 1e-12, 200)
    assert res.status == orc.OK
    assert res.iters <= orc.d_Nna(N, n, 1.0) + 1


def test_optimal_m1_equals_jacobi_m2_iterates():
    """Footnote to Thm. 3.2 and Sec. 3.4.2: optimal m = 1 and block Jacobi
    m = 2 are the same preconditioner, so PCG runs the same iterates."""
    inst = wl.small_ocp(21, 24, 4)
    r1 = orc.pcg_opt(inst.D, inst.O, inst.b, [1.0], 1e-10, 500)
    r2 = orc.pcg(inst.D, inst.O, inst.b, lambda r: orc.apply_family(inst.D, inst.O, r, 0.0, [1.0, 1.0]),
                 1e-10, 500)
    assert r1.iters == r2.iters
    assert np.allclose(r1.x, r2.x, rtol=1e-9, atol=1e-12)


def test_polycoeff_needs_fewer_iterations_than_optimal():
    """Sec. 5 finding, on the synthetic LQR family: alpha = (1, 7) at m = 2
    takes fewer PCG iterations than alpha = (1, 1)."""
    inst = wl.small_ocp(22, 30, 20)
    it_opt = orc.pcg_opt(inst.D, inst.O, inst.b, [1.0, 1.0], 1e-8, 2000).iters
    it_pc = orc.pcg_opt(inst.D, inst.O, inst.b, [1.0, 7.0], 1e-8, 2000).iters
    it_m1 = orc.pcg_opt(inst.D, inst.O, inst.b, [1.0], 1e-8, 2000).iters
    assert it_pc < it_opt < it_m1


def test_pcg_multi_rhs_columns_independent():
    inst = wl.small_llt(23, 12, 3, nrhs=3)
    for j in range(3):
        res = orc.pcg_opt(inst.D, inst.O, inst.b[:, :, j], [1.0, 7.0], 1e-10, 500)
        x = orc.direct_solve(inst.D, inst.O, inst.b[:, :, j])
        assert np.linalg.norm(res.x - x) <= 1e-6 * np.linalg.norm(x)


def test_pcg_status_paths():
    inst = wl.small_ocp(24, 10, 3)
    D, O, b = inst.D, inst.O, inst.b
    assert orc.pcg_opt(D, O, np.zeros_like(b), [1.0, 7.0], 1e-8, 10).iters == 0
    r = orc.pcg_opt(D, O, b, [1.0, 7.0], 1e-14, 1)
    assert r.status == orc.NO_CONVERGENCE and r.iters == 1
    bad = b.copy()
    bad[3, 1] = np.nan
    assert orc.pcg_opt(D, O, bad, [1.0, 7.0], 1e-8, 10).status == orc.NONFINITE
    # an indefinite S: p.q <= 0 at some step, with the identity preconditioner
    Dn = D.copy()
    Dn[5] = -Dn[5]
    rr = orc.pcg(Dn, O, b, lambda v: v.copy(), 1e-10, 200)
    assert rr.status == orc.BREAKDOWN


def test_warm_start_reduces_iterations():
    inst = wl.small_ocp(25, 40, 6)
    x = orc.direct_solve(inst.D, inst.O, inst.b)
    cold = orc.pcg_opt(inst.D, inst.O, inst.b, [1.0, 7.0], 1e-10, 500)
    warm = orc.pcg_opt(inst.D, inst.O, inst.b, [1.0, 7.0], 1e-10, 500, x0=x + 1e-9)
    assert warm.iters < cold.iters


def test_lanczos_condition_estimate_brackets_true_kappa():
    inst = wl.small_ocp(26, 8, 3)
    res = orc.pcg_opt(inst.D, inst.O, inst.b, [1.0], 1e-13, 500)
    Bk = orc.opt_blocks(inst.D, inst.O)
    N, n = 8, 3
    I = np.eye(N * n)
    Minv = np.stack([orc.apply_opt(Bk, I[:, j].reshape(N, n), [1.0]).reshape(-1) for j in range(N * n)], 1)
    A = orc.assemble(inst.D, inst.O)
    L = np.linalg.cholesky(A)
    ev = np.linalg.eigvalsh(L.T @ Minv @ L)
    est = orc.lanczos_cond(res.alphas, res.betas)
    assert est <= ev[-1] / ev[0] * (1 + 1e-6)
    assert est >= 0.5 * ev[-1] / ev[0]
