"""Spectral pins (Sec. 3): the oracle's preconditioner, built as an operator
by applying it to identity columns, must have the spectrum the paper's
lemmas fix in terms of the eigenvalues of B_l^-1 C_l."""
import json
import os

import numpy as np
import pytest

from oracle import bt_oracle as orc
from paper_2503_15269_gb300 import workloads as wl

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_counts.json")))
ZERO = 1e-9


def operator(fn, N, n):
    I = np.eye(N * n)
    return np.stack([fn(I[:, j].reshape(N, n)).reshape(-1) for j in range(N * n)], axis=1)


def eig_BlCl(D, O):
    Bd, Cd, Bl, Cl, Br, Cr = orc.splittings(D, O)
    return np.linalg.eigvals(np.linalg.solve(Bl, Cl))


def eig_sym_precond(A, Minv):
    """Eigenvalues of M^-1 A through the symmetric form L^T M^-1 L, A = L L^T."""
    L = np.linalg.cholesky(A)
    T = L.T @ Minv @ L
    return np.linalg.eigvalsh(0.5 * (T + T.T))


def cluster(vals, rel=1e-7):
    vals = np.sort(vals)
    groups = [[vals[0]]]
    for v in vals[1:]:
        if abs(v - groups[-1][-1]) <= rel * max(1.0, abs(v)):
            groups[-1].append(v)
        else:
            groups.append([v])
    return groups


@pytest.mark.parametrize("N,n", [(2, 2), (3, 2), (4, 3), (5, 3), (6, 2), (7, 2), (8, 1)])
def test_lemma33_spectrum_of_BlCl(N, n):
    """ceil(N/2) n exact zeros; the other eigenvalues real and in (0, 1)
    (Lemma 3.3; zero count from Table I)."""
    inst = wl.small_ocp(10, N, n)
    ev = eig_BlCl(inst.D, inst.O)
    zeros = np.abs(ev) < ZERO
    assert zeros.sum() == -(-N // 2) * n
    nz = ev[~zeros]
    assert np.all(np.abs(nz.imag) < 1e-9)
    assert np.all((nz.real > 0) & (nz.real < 1))


@pytest.mark.parametrize("a", [0.0, 0.2, 1.0 / 3.0, 0.4, 0.5, 0.7, 1.0])
@pytest.mark.parametrize("m", [1, 2, 3])
@pytest.mark.parametrize("N", [4, 5])
def test_lemma32_eigenvalues_of_MinvA(a, m, N):
    """eig(_{ab}M_m^-1 A) = {1 - f_{a+-}(lam)^m : lam != 0}, plus n ones for
    odd N (Lemmas 3.1, 3.2 and Thm. 3.2's counting)."""
    n = 2
    inst = wl.small_llt(11, N, n)
    lam = np.sort(eig_BlCl(inst.D, inst.O).real)
    lam = lam[np.abs(lam) > ZERO]
    pred = np.concatenate([1 - orc.f_a(lam, a, +1) ** m, 1 - orc.f_a(lam, a, -1) ** m])
    if N % 2 == 1:
        pred = np.concatenate([pred, np.ones(n)])
    A = orc.assemble(inst.D, inst.O)
    Minv = operator(lambda r: orc.apply_family(inst.D, inst.O, r, a, [1.0] * m), N, n)
    got = eig_sym_precond(A, Minv)
    assert np.allclose(np.sort(got), np.sort(pred), atol=1e-8)


@pytest.mark.parametrize("alpha", [(1.0, 7.0), (1.0, 0.5, 2.0), (1.0, 1.0, 1.0, 7.0)])
def test_polycoeff_spectrum_and_count(alpha):
    """With coefficients alpha at a = 1, M^-1 A v = (1 - lam) q(lam) v with
    q(t) = sum alpha_j t^j (Lemma 3.2's proof with the sum weighted), and the
    distinct count stays N n / 2 or floor(N/2) n + 1 (Thm. 3.3)."""
    for N in (6, 7):
        n = 2
        inst = wl.small_ocp(12, N, n)
        lam = np.sort(eig_BlCl(inst.D, inst.O).real)
        lam = lam[np.abs(lam) > ZERO]
        q = sum(aj * lam ** j for j, aj in enumerate(alpha))
        pred = np.concatenate([(1 - lam) * q, (1 - lam) * q])
        if N % 2 == 1:
            pred = np.concatenate([pred, np.ones(n)])
        A = orc.assemble(inst.D, inst.O)
        Bk = orc.opt_blocks(inst.D, inst.O)
        Minv = operator(lambda r: orc.apply_opt(Bk, r, alpha), N, n)
        got = eig_sym_precond(A, Minv)
        assert np.allclose(np.sort(got), np.sort(pred), atol=1e-8)
        assert len(cluster(got)) == orc.d_Nna(N, n, 1.0)


@pytest.mark.parametrize("N,n", [(4, 3), (5, 3), (6, 2), (7, 2)])
def test_thm32_distinct_count_and_pairs(N, n):
    """a = 1: d_Nna distinct eigenvalues, every value in (0,1) twice, n ones
    for odd N (Table I, Thm. 3.2).  a in [0,1): the larger count."""
    inst = wl.small_llt(13, N, n)
    A = orc.assemble(inst.D, inst.O)
    for m in (1, 2, 3):
        Bk = orc.opt_blocks(inst.D, inst.O)
        got = eig_sym_precond(A, operator(lambda r: orc.apply_opt(Bk, r, [1.0] * m), N, n))
        groups = cluster(got)
        assert len(groups) == orc.d_Nna(N, n, 1.0)
        ones = [g for g in groups if abs(g[0] - 1.0) < 1e-9]
        inner = [g for g in groups if abs(g[0] - 1.0) >= 1e-9]
        assert all(len(g) == 2 for g in inner)
        assert (len(ones[0]) if ones else 0) == (n if N % 2 == 1 else 0)
    got = eig_sym_precond(A, operator(lambda r: orc.apply_family(inst.D, inst.O, r, 0.5, [1.0, 1.0]), N, n))
    assert len(cluster(got)) == orc.d_Nna(N, n, 0.5)


def test_golden_counts():
    for row in GOLD["g_a"]:
        assert orc.g_a(row["m"], row["a"]) == row["value"]
    for row in GOLD["d_Nna"]:
        assert orc.d_Nna(row["N"], row["n"], row["a"]) == row["value"]


@pytest.mark.parametrize("N", [6, 7])
def test_table1_rows(N):
    """Counts of exact zeros / ones / distinct values in (0,1) for the
    matrices of Table I, evaluated from the printed formulas."""
    n = 2
    k = N // 2 if N % 2 == 0 else (N + 1) // 2
    rows = GOLD["table1"]["even" if N % 2 == 0 else "odd"]
    ev_ = lambda s: eval(s, {}, {"k": k, "n": n})
    inst = wl.small_ocp(14, N, n)
    A = orc.assemble(inst.D, inst.O)
    G, H = orc.GH_dense(inst.D, inst.O, 1.0)
    mats = {"BlCl": eig_BlCl(inst.D, inst.O), "H_opt": np.linalg.eigvals(H),
            "G_opt_A": np.linalg.eigvals(G @ A),
            "M_A": np.linalg.eigvals((np.eye(N * n) + H) @ G @ A)}
    for name, ev in mats.items():
        ev = ev.real
        spec = rows[name]
        assert (np.abs(ev) < ZERO).sum() == ev_(spec["zeros"]), name
        assert (np.abs(ev - 1) < 1e-9).sum() == ev_(spec["ones"]), name
        inner = ev[(np.abs(ev) >= ZERO) & (np.abs(ev - 1) >= 1e-9)]
        assert np.all((inner > 0) & (inner < 1)), name
        groups = cluster(inner, 1e-6)
        assert len(groups) == ev_(spec["distinct_open01"]), name
        if spec.get("paired"):
            assert all(len(g) == 2 for g in groups), name


@pytest.mark.parametrize("a", [0.0, 0.1, 1.0 / 3.0, 0.5, 0.9, 1.0])
def test_lemma34_ranges(a):
    """rho(H_ab) = max over the spectrum of max(|f_{a+}|, |f_{a-}|) < 1 and
    the eigenvalues of G_ab A lie in the stated interval (Lemma 3.4, Table
    of the appendix).  The lemma's endpoints are suprema (open ends)."""
    N, n = 6, 3
    inst = wl.small_ocp(15, N, n)
    lam = eig_BlCl(inst.D, inst.O).real
    lam = lam[np.abs(lam) > ZERO]
    G, H = orc.GH_dense(inst.D, inst.O, a)
    A = orc.assemble(inst.D, inst.O)
    rho = np.abs(np.linalg.eigvals(H)).max()
    pred = max(np.abs(orc.f_a(lam, a, 1)).max(), np.abs(orc.f_a(lam, a, -1)).max())
    assert abs(rho - pred) < 1e-9 and rho < 1
    sup = 2 - 2 * a if a <= 1.0 / 3.0 else 1 + (1 - a) ** 2 / (4 * a)
    evGA = np.linalg.eigvals(G @ A).real
    assert evGA.min() > 0 and evGA.max() <= sup + 1e-12


@pytest.mark.parametrize("a", [-0.5, 1.5])
def test_lemma34_outside_unit_interval_diverges(a):
    """For a outside [0,1] some lam in [0,1) gives rho(H_ab) > 1; with the
    largest lam of a typical instance near 1 this shows up directly."""
    N, n = 8, 3
    inst = wl.small_ocp(16, N, n)
    lam = eig_BlCl(inst.D, inst.O).real
    lmax = lam.max()
    thr = 1.0 / a if a > 1 else 1.0 / (1 - a) ** 2
    assert lmax > thr
    _, H = orc.GH_dense(inst.D, inst.O, a)
    assert np.abs(np.linalg.eigvals(H)).max() > 1


@pytest.mark.parametrize("a", [0.0, 0.25, 1.0 / 3.0, 0.5, 0.75, 1.0])
@pytest.mark.parametrize("m", [1, 2, 3, 4])
def test_thm31_preconditioner_is_spd(a, m):
    N, n = 5, 3
    inst = wl.small_ocp(17, N, n)
    Minv = operator(lambda r: orc.apply_family(inst.D, inst.O, r, a, [1.0] * m), N, n)
    assert np.abs(Minv - Minv.T).max() <= 1e-10 * np.abs(Minv).max()
    np.linalg.cholesky(0.5 * (Minv + Minv.T))


@pytest.mark.parametrize("alpha", [(1.0, 7.0), (1.0, 0.0, 3.0), (1.0, 0.5, 2.0, 7.0)])
def test_polycoeff_nonnegative_alpha_is_spd(alpha):
    """Reading: at a = 1 the eigenvalues of H_opt are in [0,1), so alpha_j >= 0
    keeps q > 0 and M^-1 SPD."""
    N, n = 6, 2
    inst = wl.small_llt(18, N, n)
    Bk = orc.opt_blocks(inst.D, inst.O)
    Minv = operator(lambda r: orc.apply_opt(Bk, r, alpha), N, n)
    assert np.abs(Minv - Minv.T).max() <= 1e-10 * np.abs(Minv).max()
    np.linalg.cholesky(0.5 * (Minv + Minv.T))


def test_remark_larger_m_moves_spectrum_toward_one():
    N, n = 6, 2
    inst = wl.small_ocp(19, N, n)
    A = orc.assemble(inst.D, inst.O)
    Bk = orc.opt_blocks(inst.D, inst.O)
    prev = None
    for m in (1, 2, 3, 4):
        ev = eig_sym_precond(A, operator(lambda r: orc.apply_opt(Bk, r, [1.0] * m), N, n))
        dist = np.abs(1 - ev).max()
        if prev is not None:
            assert dist < prev
        prev = dist
