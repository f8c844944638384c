"""Differentiable batched solve (hand-written adjoint) against the oracle's
adjoint, dense torch autograd at N = 8 and central finite differences."""
import numpy as np
import pytest
import torch

from oracle import bt_oracle as orc
from paper_2503_15269_gb300 import binding as bb
from paper_2503_15269_gb300 import workloads as wl

from _util import cond_estimate, dev, host, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2503_15269_gb300 import build
    build.build()
    bb.lib()


def packed(insts):
    Ns, ns, d_off, o_off, v_off, D, O, b = wl.pack_batch(insts)
    return Ns, ns, d_off, o_off, v_off, dev(D).requires_grad_(), dev(O).requires_grad_(), dev(b).requires_grad_()


def unpack_grads(insts, d_off, o_off, v_off, gD, gO, gb):
    out = []
    for k, inst in enumerate(insts):
        N, n = inst.N, inst.n
        out.append((gb[v_off[k]:v_off[k] + N * n].reshape(N, n),
                    gD[d_off[k]:d_off[k] + N * n * n].reshape(N, n, n),
                    gO[o_off[k]:o_off[k] + (N - 1) * n * n].reshape(N - 1, n, n)))
    return out


@pytest.mark.parametrize("precision,tol,gtol", [(bb.BT_FP64, 1e-13, 1e-9), (bb.BT_MIXED, 1e-13, 1e-8)])
def test_adjoint_matches_oracle(precision, tol, gtol):
    from paper_2503_15269_gb300.autograd import bt_solve
    insts = [wl.small_ocp(80 + k, N, n) for k, (N, n) in enumerate([(8, 3), (12, 6), (5, 2), (20, 4)])]
    Ns, ns, d_off, o_off, v_off, D, O, b = packed(insts)
    w = torch.randn(b.shape, dtype=torch.float64, device=b.device, generator=torch.Generator(device=b.device).manual_seed(0))
    x = bt_solve(D, O, b, Ns, ns, d_off, o_off, precision=precision, tol=tol)
    (x * w).sum().backward()
    grads = unpack_grads(insts, d_off, o_off, v_off, host(D.grad).ravel(), host(O.grad).ravel(), host(b.grad))
    wn = host(w)
    for k, inst in enumerate(insts):
        xk = host(x)[v_off[k]:v_off[k] + inst.N * inst.n].reshape(inst.N, inst.n)
        xr = orc.direct_solve(inst.D, inst.O, inst.b)
        assert rel(xk, xr) <= gtol
        g, gD, gO = orc.adjoint(inst.D, inst.O, xr, wn[v_off[k]:v_off[k] + inst.N * inst.n].reshape(inst.N, inst.n))
        assert rel(grads[k][0], g) <= gtol
        assert rel(grads[k][1], gD) <= gtol
        assert rel(grads[k][2], gO) <= gtol


def test_adjoint_matches_dense_autograd_N8():
    from paper_2503_15269_gb300.autograd import bt_solve
    inst = wl.small_ocp(90, 8, 4)
    Ns, ns, d_off, o_off, v_off, D, O, b = packed([inst])
    x = bt_solve(D, O, b, Ns, ns, d_off, o_off, precision=bb.BT_FP64, tol=1e-14, maxit=1000)
    w = torch.linspace(-1, 1, b.numel(), dtype=torch.float64, device=b.device)
    (x * w).sum().backward()
    # dense reference on the CPU
    Dt = torch.tensor(inst.D, requires_grad=True)
    Ot = torch.tensor(inst.O, requires_grad=True)
    bt = torch.tensor(inst.b.reshape(-1), requires_grad=True)
    N, n = 8, 4
    S = torch.zeros(N * n, N * n, dtype=torch.float64)
    for i in range(N):
        S = S.index_put((torch.arange(i * n, (i + 1) * n)[:, None], torch.arange(i * n, (i + 1) * n)[None, :]), Dt[i])
    for i in range(N - 1):
        r = torch.arange(i * n, (i + 1) * n)
        c = torch.arange((i + 1) * n, (i + 2) * n)
        S = S.index_put((r[:, None], c[None, :]), Ot[i])
        S = S.index_put((c[:, None], r[None, :]), Ot[i].T)
    xt = torch.linalg.solve(S, bt)
    (xt * w.cpu()).sum().backward()
    assert rel(host(x), xt.detach().numpy()) <= 1e-11
    assert rel(host(b.grad), bt.grad.numpy()) <= 1e-10
    assert rel(host(D.grad).reshape(N, n, n), Dt.grad.numpy()) <= 1e-10
    assert rel(host(O.grad).reshape(N - 1, n, n), Ot.grad.numpy()) <= 1e-10


def test_adjoint_central_differences():
    from paper_2503_15269_gb300.autograd import bt_solve
    inst = wl.small_ocp(91, 8, 3)
    Ns, ns, d_off, o_off, v_off, D, O, b = packed([inst])
    rng = np.random.default_rng(4)
    w = dev(rng.standard_normal(b.numel()))
    x = bt_solve(D, O, b, Ns, ns, d_off, o_off, precision=bb.BT_FP64, tol=1e-14, maxit=1000)
    (x * w).sum().backward()
    dD = rng.standard_normal(inst.D.shape)
    dD = 0.5 * (dD + dD.transpose(0, 2, 1))
    dO = rng.standard_normal(inst.O.shape)
    db = rng.standard_normal(inst.b.shape)
    h = 1e-6

    def f(sign):
        with torch.no_grad():
            xx = bt_solve(dev((inst.D + sign * h * dD).ravel()), dev((inst.O + sign * h * dO).ravel()),
                          dev((inst.b + sign * h * db).ravel()), Ns, ns, d_off, o_off, precision=bb.BT_FP64,
                          tol=1e-14, maxit=1000)
        return float((xx * w).sum())

    fd = (f(+1) - f(-1)) / (2 * h)
    an = float(np.sum(host(D.grad) * dD.ravel()) + np.sum(host(O.grad) * dO.ravel()) + np.sum(host(b.grad) * db.ravel()))
    assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


def test_config4_forward_backward_mixed():
    """256 instances, N = 256, n = 24 (input size 8): mixed forward and
    adjoint at the benchmark's tol = 1e-8, every instance by its forward and
    adjoint residuals; then at tol = min(1e-8, 1e-8 / cond(S)) over the
    sampled instances (cond from the oracle's Lanczos estimate, about 6e2),
    sampled x, grad b, grad D and grad O against the oracle's direct solve and
    adjoint at <= 1e-8."""
    from paper_2503_15269_gb300.autograd import bt_solve
    insts = wl.config4()
    Ns, ns, d_off, o_off, v_off, D, O, b = packed(insts)
    w = dev(np.random.default_rng(5).standard_normal(b.numel()))
    x = bt_solve(D, O, b, Ns, ns, d_off, o_off, precision=bb.BT_MIXED, tol=1e-8)
    (x * w).sum().backward()
    xs, gb = host(x), host(b.grad)
    wn = host(w)
    for k in range(len(insts)):
        inst = insts[k]
        sl = slice(v_off[k], v_off[k] + inst.N * inst.n)
        xk = xs[sl].reshape(inst.N, inst.n)
        assert np.linalg.norm(orc.spmv(inst.D, inst.O, xk) - inst.b) <= 1e-8 * np.linalg.norm(inst.b)
        gk = gb[sl].reshape(inst.N, inst.n)
        wk = wn[sl].reshape(inst.N, inst.n)
        assert np.linalg.norm(orc.spmv(inst.D, inst.O, gk) - wk) <= 1e-8 * np.linalg.norm(wk)
    samples = (0, 77, 255)
    cond = max(cond_estimate(insts[k].D, insts[k].O, insts[k].b) for k in samples)
    tol = min(1e-8, 1e-8 / cond)
    D.grad = O.grad = b.grad = None
    x = bt_solve(D, O, b, Ns, ns, d_off, o_off, precision=bb.BT_MIXED, tol=tol)
    (x * w).sum().backward()
    xs, gb = host(x), host(b.grad)
    gDall, gOall = host(D.grad).ravel(), host(O.grad).ravel()
    for k in samples:
        inst = insts[k]
        sl = slice(v_off[k], v_off[k] + inst.N * inst.n)
        xr = orc.direct_solve(inst.D, inst.O, inst.b)
        g, gD, gO = orc.adjoint(inst.D, inst.O, xr, wn[sl].reshape(inst.N, inst.n))
        gDk = gDall[d_off[k]:d_off[k] + inst.N * inst.n ** 2].reshape(gD.shape)
        gOk = gOall[o_off[k]:o_off[k] + (inst.N - 1) * inst.n ** 2].reshape(gO.shape)
        assert rel(xs[sl].reshape(inst.N, inst.n), xr) <= 1e-8
        assert rel(gb[sl].reshape(inst.N, inst.n), g) <= 1e-8
        assert rel(gDk, gD) <= 1e-8
        assert rel(gOk, gO) <= 1e-8
