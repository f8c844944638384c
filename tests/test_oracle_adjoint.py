"""Pins for the oracle adjoint: central finite differences (step 1e-6) and
dense autograd through torch.linalg.solve (CPU, float64) at N = 8."""
import numpy as np
import pytest
import torch

from oracle import bt_oracle as orc
from paper_2503_15269_gb300 import workloads as wl


def loss_and_grads(D, O, b, w):
    x = orc.direct_solve(D, O, b)
    return float(np.sum(w * x)), x


def test_adjoint_matches_dense_autograd():
    inst = wl.small_ocp(30, 8, 4)
    D, O, b = inst.D, inst.O, inst.b
    w = np.random.default_rng(1).standard_normal(b.shape)
    x = orc.direct_solve(D, O, b)
    g, gD, gO = orc.adjoint(D, O, x, w)
    Dt = torch.tensor(D, requires_grad=True)
    Ot = torch.tensor(O, requires_grad=True)
    bt = torch.tensor(b.reshape(-1), requires_grad=True)
    N, n = D.shape[0], D.shape[1]
    rows = []
    for i in range(N):
        row = []
        for j in range(N):
            if j == i:
                row.append(Dt[i])
            elif j == i + 1:
                row.append(Ot[i])
            elif j == i - 1:
                row.append(Ot[j].T)
            else:
                row.append(torch.zeros(n, n, dtype=torch.float64))
        rows.append(torch.cat(row, 1))
    S = torch.cat(rows, 0)
    xt = torch.linalg.solve(S, bt)
    (xt * torch.tensor(w.reshape(-1))).sum().backward()
    assert np.allclose(g.reshape(-1), bt.grad.numpy(), rtol=1e-9, atol=1e-12)
    assert np.allclose(gD, Dt.grad.numpy(), rtol=1e-9, atol=1e-12)
    assert np.allclose(gO, Ot.grad.numpy(), rtol=1e-9, atol=1e-12)


def test_adjoint_matches_central_differences():
    inst = wl.small_ocp(31, 8, 3)
    D, O, b = inst.D, inst.O, inst.b
    rng = np.random.default_rng(2)
    w = rng.standard_normal(b.shape)
    x = orc.direct_solve(D, O, b)
    g, gD, gO = orc.adjoint(D, O, x, w)
    h = 1e-6
    # symmetric perturbation of D (S stays SPD), random O and b directions
    dD = rng.standard_normal(D.shape)
    dD = 0.5 * (dD + dD.transpose(0, 2, 1))
    dO = rng.standard_normal(O.shape)
    db = rng.standard_normal(b.shape)
    fp, _ = loss_and_grads(D + h * dD, O + h * dO, b + h * db, w)
    fm, _ = loss_and_grads(D - h * dD, O - h * dO, b - h * db, w)
    fd = (fp - fm) / (2 * h)
    an = np.sum(gD * dD) + np.sum(gO * dO) + np.sum(g * db)
    assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))
