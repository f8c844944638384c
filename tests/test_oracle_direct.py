"""Pins for the oracle's direct solve and SpMV (Sec. 4.3, Eq. 1) against
numpy's dense solver and the generator's own factors."""
import numpy as np
import pytest

from oracle import bt_oracle as orc
from paper_2503_15269_gb300 import workloads as wl


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 8])
@pytest.mark.parametrize("n", [1, 2, 3, 6])
def test_direct_solve_matches_dense(N, n):
    inst = wl.small_llt(0, N, n)
    S = orc.assemble(inst.D, inst.O)
    x = orc.direct_solve(inst.D, inst.O, inst.b)
    ref = np.linalg.solve(S, inst.b.reshape(-1)).reshape(N, n)
    assert np.allclose(x, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("N,n", [(4, 3), (7, 5), (9, 2)])
def test_direct_solve_multi_rhs(N, n):
    inst = wl.small_ocp(1, N, n)
    rhs = np.random.default_rng(3).standard_normal((N, n, 4))
    x = orc.direct_solve(inst.D, inst.O, rhs)
    S = orc.assemble(inst.D, inst.O)
    ref = np.linalg.solve(S, rhs.reshape(N * n, 4)).reshape(N, n, 4)
    assert np.allclose(x, ref, rtol=1e-10, atol=1e-12)


def test_spmv_matches_dense():
    inst = wl.small_ocp(2, 9, 4)
    x = np.random.default_rng(0).standard_normal((9, 4))
    S = orc.assemble(inst.D, inst.O)
    assert np.allclose(orc.spmv(inst.D, inst.O, x).reshape(-1), S @ x.reshape(-1), rtol=1e-13, atol=1e-13)


def test_assemble_is_LLt_for_llt_family():
    """The llt generator promises S = L L^T with L lower block-bidiagonal
    (diag L_i, sub-diagonal M_i); rebuild that L densely and compare."""
    inst = wl.config0()
    N, n = inst.N, inst.n
    L = np.zeros((N * n, N * n))
    for i in range(N):
        L[i * n:(i + 1) * n, i * n:(i + 1) * n] = inst.L[i]
        if i < N - 1:
            L[(i + 1) * n:(i + 2) * n, i * n:(i + 1) * n] = inst.M[i]
    assert np.allclose(orc.assemble(inst.D, inst.O), L @ L.T, rtol=1e-14, atol=1e-13)
    S = orc.assemble(inst.D, inst.O)
    assert np.allclose(S, S.T)
    assert np.linalg.eigvalsh(S).min() > 0


def test_ocp_instance_is_schur_complement():
    """The ocp generator's closed form equals C G^-1 C^T assembled densely
    from the LQR data (same seed, redrawn here)."""
    N, n, m = 5, 3, 2
    rng = np.random.Generator(np.random.PCG64(12345))
    inst = wl.ocp_instance(rng, N, n, m)
    rng = np.random.Generator(np.random.PCG64(12345))
    A = np.eye(n) + 0.05 * rng.standard_normal((N - 1, n, n))
    B = 0.05 * rng.standard_normal((N - 1, n, m))
    Q = rng.uniform(1.0, 10.0, (N, n))
    R = rng.uniform(0.1, 1.0, (N - 1, m))
    nv = N * n + (N - 1) * m
    xcol = lambda k: k * (n + m)
    ucol = lambda k: k * (n + m) + n
    C = np.zeros((N * n, nv))
    Gd = np.zeros(nv)
    for k in range(N):
        Gd[xcol(k):xcol(k) + n] = Q[k]
        if k < N - 1:
            Gd[ucol(k):ucol(k) + m] = R[k]
    C[0:n, xcol(0):xcol(0) + n] = np.eye(n)
    for k in range(N - 1):
        r = slice((k + 1) * n, (k + 2) * n)
        C[r, xcol(k + 1):xcol(k + 1) + n] = np.eye(n)
        C[r, xcol(k):xcol(k) + n] = -A[k]
        C[r, ucol(k):ucol(k) + m] = -B[k]
    S = C @ np.diag(1.0 / Gd) @ C.T
    assert np.allclose(orc.assemble(inst.D, inst.O), S, rtol=1e-13, atol=1e-14)


def test_block_cholesky_reports_first_non_spd_block():
    inst = wl.small_llt(4, 6, 3)
    D = inst.D.copy()
    D[3] = -np.eye(3)
    _, _, st, blk = orc.block_cholesky(D, inst.O)
    assert st == orc.NOT_SPD and blk <= 3
