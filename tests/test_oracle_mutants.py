"""Planted mistakes in the oracle (on the CPU) must be caught by the pins:
each mutant below is a plausible slip -- a dropped term, a wrong sign, a
transposed operand, a shifted index -- and at least one independent check
(dense definition or footnote identity) must reject it."""
import numpy as np
import pytest

from oracle import bt_oracle as orc
from paper_2503_15269_gb300 import workloads as wl


def mut_drop_ET(B, r):
    N = B.Dinv.shape[0]
    y = np.zeros_like(r)
    for i in range(N):
        y[i] = B.Dinv[i] @ r[i]
        if i < N - 1:
            y[i] -= B.E[i] @ r[i + 1]
    return y


def mut_sign_E(B, r):
    N = B.Dinv.shape[0]
    y = np.zeros_like(r)
    for i in range(N):
        y[i] = B.Dinv[i] @ r[i]
        if i < N - 1:
            y[i] += B.E[i] @ r[i + 1]
        if i > 0:
            y[i] -= B.E[i - 1].T @ r[i - 1]
    return y


def mut_transpose_E(B, r):
    N = B.Dinv.shape[0]
    y = np.zeros_like(r)
    for i in range(N):
        y[i] = B.Dinv[i] @ r[i]
        if i < N - 1:
            y[i] -= B.E[i].T @ r[i + 1]
        if i > 0:
            y[i] -= B.E[i - 1] @ r[i - 1]
    return y


def mut_H_shift(B, y):
    N = B.Dinv.shape[0]
    w = np.zeros_like(y)
    for i in range(N):
        w[i] = B.Hd[i] @ y[i]
        if i + 2 < N:
            w[i] += B.Hu[i] @ y[i + 2]
        if i - 2 >= 0:
            w[i] += B.Hl[i - 2].T @ y[i - 2]
    return w


@pytest.mark.parametrize("which", ["drop_ET", "sign_E", "transpose_E", "H_shift"])
def test_mutant_is_rejected(which, monkeypatch):
    inst = wl.small_llt(40, 6, 3)
    r = np.random.default_rng(0).standard_normal((6, 3))
    ref = orc.apply_jacobi_sweeps(inst.D, inst.O, r, 2)
    good = orc.apply_opt(orc.opt_blocks(inst.D, inst.O), r, [1.0, 1.0])
    assert np.allclose(good, ref, rtol=1e-9, atol=1e-10)
    if which == "H_shift":
        monkeypatch.setattr(orc, "apply_H_opt", mut_H_shift)
    else:
        monkeypatch.setattr(orc, "apply_G_opt", {"drop_ET": mut_drop_ET, "sign_E": mut_sign_E,
                                                 "transpose_E": mut_transpose_E}[which])
    bad = orc.apply_opt(orc.opt_blocks(inst.D, inst.O), r, [1.0, 1.0])
    assert not np.allclose(bad, ref, rtol=1e-6, atol=1e-8)


def test_mutant_pcg_sign_is_rejected():
    """A PCG with beta's sign flipped no longer reaches the direct solution."""
    inst = wl.small_ocp(41, 10, 3)
    Bk = orc.opt_blocks(inst.D, inst.O)
    x = orc.direct_solve(inst.D, inst.O, inst.b)

    def bad_pcg(D, O, b, minv, tol, maxit):
        xx = np.zeros_like(b); r = b.copy(); z = minv(r); p = z.copy(); rho = np.vdot(r, z)
        for _ in range(maxit):
            q = orc.spmv(D, O, p); al = rho / np.vdot(p, q); xx += al * p; r -= al * q
            z = minv(r); rn = np.vdot(r, z); p = z - (rn / rho) * p; rho = rn
        return xx

    xb = bad_pcg(inst.D, inst.O, inst.b, lambda v: orc.apply_opt(Bk, v, [1.0, 7.0]), 1e-10,
                 orc.pcg_opt(inst.D, inst.O, inst.b, [1.0, 7.0], 1e-10, 500).iters)
    assert np.linalg.norm(xb - x) > 1e-4 * np.linalg.norm(x)
