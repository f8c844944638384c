"""Pins for the preconditioner blocks: the Sec. 4.1 closed form against the
dense multi-splitting definition (Sec. 3.1), the general-a reading against
the same definition, and the footnote identity of Thm. 3.2 (a second,
independent construction)."""
import numpy as np
import pytest

from oracle import bt_oracle as orc
from paper_2503_15269_gb300 import workloads as wl

CASES = [(2, 2), (3, 2), (4, 3), (5, 3), (6, 2), (7, 3)]


def dense_from_opt(Bk, N, n):
    G = np.zeros((N * n, N * n))
    H = np.zeros((N * n, N * n))
    blk = lambda i, j: (slice(i * n, (i + 1) * n), slice(j * n, (j + 1) * n))
    for i in range(N):
        G[blk(i, i)] = Bk.Dinv[i]
        H[blk(i, i)] = Bk.Hd[i]
    for i in range(N - 1):
        G[blk(i, i + 1)] = -Bk.E[i]
        G[blk(i + 1, i)] = -Bk.E[i].T
    for i in range(N - 2):
        H[blk(i, i + 2)] = Bk.Hu[i]
        H[blk(i + 2, i)] = Bk.Hl[i]
    return G, H


@pytest.mark.parametrize("N,n", CASES)
def test_opt_closed_form_matches_definition(N, n):
    inst = wl.small_ocp(0, N, n)
    G, H = orc.GH_dense(inst.D, inst.O, 1.0)
    Gc, Hc = dense_from_opt(orc.opt_blocks(inst.D, inst.O), N, n)
    sc = np.abs(G).max()
    assert np.abs(G - Gc).max() <= 1e-11 * sc
    assert np.abs(H - Hc).max() <= 1e-11 * max(1.0, np.abs(H).max())


@pytest.mark.parametrize("a", [0.0, 0.2, 1.0 / 3.0, 0.5, 0.8, 1.0])
def test_G_A_plus_H_is_identity(a):
    """G_ab A + H_ab = I for every (a, b) with 2a + b = 1 (proof of Lemma 3.1)."""
    inst = wl.small_llt(1, 5, 3)
    A = orc.assemble(inst.D, inst.O)
    G, H = orc.GH_dense(inst.D, inst.O, a)
    assert np.allclose(G @ A + H, np.eye(A.shape[0]), atol=1e-10)


@pytest.mark.parametrize("a", [0.0, 0.25, 0.5, 0.75, 1.0])
@pytest.mark.parametrize("alpha", [(1.0,), (1.0, 1.0), (1.0, 7.0), (1.0, 0.5, 2.0)])
def test_family_apply_matches_dense_polynomial(a, alpha):
    N, n = 6, 3
    inst = wl.small_ocp(2, N, n)
    G, H = orc.GH_dense(inst.D, inst.O, a)
    r = np.random.default_rng(5).standard_normal((N, n))
    Minv = np.zeros_like(G)
    Hp = np.eye(G.shape[0])
    for aj in alpha:
        Minv += aj * Hp
        Hp = Hp @ H
    ref = (Minv @ G @ r.reshape(-1)).reshape(N, n)
    z = orc.apply_family(inst.D, inst.O, r, a, alpha)
    assert np.allclose(z, ref, rtol=1e-10, atol=1e-11 * np.abs(ref).max())
    if a == 1.0:
        z2 = orc.apply_opt(orc.opt_blocks(inst.D, inst.O), r, alpha)
        assert np.allclose(z2, ref, rtol=1e-10, atol=1e-11 * np.abs(ref).max())


@pytest.mark.parametrize("N,n", CASES + [(16, 6)])
@pytest.mark.parametrize("m", [1, 2, 3])
def test_footnote_identity_opt_equals_2m_jacobi(N, n, m):
    """_{1,-1}M_m^-1 = _{0,1}M_{2m}^-1 (footnote to Thm. 3.2)."""
    inst = wl.small_llt(3, N, n)
    r = np.random.default_rng(N * 10 + n).standard_normal((N, n))
    z1 = orc.apply_opt(orc.opt_blocks(inst.D, inst.O), r, [1.0] * m)
    z2 = orc.apply_jacobi_sweeps(inst.D, inst.O, r, m)
    assert np.allclose(z1, z2, rtol=1e-9, atol=1e-10 * np.abs(z2).max())


def test_G_opt_is_stair_combination():
    """G_opt = B_d^-1 (2 B_d - A) B_d^-1, i.e. B_l^-1 + B_r^-1 - B_d^-1."""
    inst = wl.small_ocp(3, 5, 2)
    Bd, Cd, Bl, Cl, Br, Cr = orc.splittings(inst.D, inst.O)
    A = orc.assemble(inst.D, inst.O)
    Bdi = np.linalg.inv(Bd)
    G, _ = orc.GH_dense(inst.D, inst.O, 1.0)
    assert np.allclose(G, Bdi @ (2 * Bd - A) @ Bdi, atol=1e-11)
    HJ = Bdi @ Cd
    _, H = orc.GH_dense(inst.D, inst.O, 1.0)
    assert np.allclose(H, HJ @ HJ, atol=1e-11)


@pytest.mark.parametrize("N", [3, 4, 5, 6])
def test_splittings_are_p_regular(N):
    """Lemmas of Sec. 2.3: B_d + C_d is SPD; sym(B_l + C_l) = sym(B_r + C_r) = B_d."""
    inst = wl.small_llt(5, N, 3)
    Bd, Cd, Bl, Cl, Br, Cr = orc.splittings(inst.D, inst.O)
    np.linalg.cholesky(Bd + Cd)
    sym = lambda X: 0.5 * (X + X.T)
    assert np.allclose(sym(Bl + Cl), Bd, atol=1e-12)
    assert np.allclose(sym(Br + Cr), Bd, atol=1e-12)
    A = orc.assemble(inst.D, inst.O)
    for B, C in ((Bd, Cd), (Bl, Cl), (Br, Cr)):
        assert np.allclose(B - C, A)


def test_opt_block_sparsity():
    """H_opt has zero +-1 block diagonals; G_opt is block tridiagonal."""
    inst = wl.small_ocp(4, 7, 2)
    G, H = orc.GH_dense(inst.D, inst.O, 1.0)
    n = 2
    for i in range(6):
        assert np.abs(H[i * n:(i + 1) * n, (i + 1) * n:(i + 2) * n]).max() < 1e-12
        assert np.abs(H[(i + 1) * n:(i + 2) * n, i * n:(i + 1) * n]).max() < 1e-12
    for i in range(4):
        assert np.abs(G[i * n:(i + 1) * n, (i + 3) * n:(i + 4) * n]).max() < 1e-12
