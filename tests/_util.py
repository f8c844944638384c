"""Helpers shared by the GPU tests (marshalling, and the oracle-side condition estimate)."""
import numpy as np

from paper_2503_15269_gb300 import binding as bb


def dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda:0")


def host(t):
    return t.detach().cpu().numpy()


class Single:
    """One instance on the device: setup + entry points, raising on error."""

    def __init__(self, inst, m=2, alpha=None, precision=bb.BT_FP64, **kw):
        self.inst = inst
        self.D = dev(inst.D)
        self.O = dev(inst.O if inst.O.size else np.zeros((1, inst.n, inst.n)))
        self.params, self._keep = bb.make_params(m=m, alpha=alpha, precision=precision, **kw)
        self.st, self.h = bb.bt_setup(inst.N, inst.n, self.D, self.O, self.params)

    def ok(self):
        assert self.st == bb.BT_OK, bb.status_string(self.st)
        return self

    def apply(self, r):
        z = dev(np.zeros(r.size))
        st = bb.bt_apply_precond(self.h, dev(r.reshape(-1)), z)
        assert st == bb.BT_OK, bb.status_string(st)
        return host(z).reshape(r.shape)

    def spmv(self, x, f32=False):
        y = dev(np.zeros(x.size))
        st = (bb.bt_spmv_f32 if f32 else bb.bt_spmv)(self.h, dev(x.reshape(-1)), y)
        assert st == bb.BT_OK, bb.status_string(st)
        return host(y).reshape(x.shape)

    def solve(self, b, tol, maxit, x0=None):
        x = dev(np.zeros(b.size) if x0 is None else x0.reshape(-1))
        st, it = bb.bt_pcg_solve(self.h, dev(b.reshape(-1)), x, tol, maxit)
        return st, it, host(x).reshape(b.shape)

    def info(self):
        return bb.bt_solve_info(self.h, 0)

    def close(self):
        if self.h:
            bb.bt_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def maxrel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def cond_estimate(D, O, b, maxit=20000):
    """kappa(S) of one system, from the oracle: the extreme Ritz values of
    the Lanczos tridiagonal of an unpreconditioned CG run (M = I) on b to a
    relative residual of 1e-12 (oracle.lanczos_cond, textbook relation).
    The relative error of a solve stopped at relative residual tol is at
    most kappa(S) * tol."""
    from oracle import bt_oracle as orc
    res = orc.pcg(D, O, b, lambda r: r, 1e-12, maxit)
    return orc.lanczos_cond(res.alphas, res.betas)


def ill_conditioned(inst, row, decades, seed):
    """Congruence S' = P^T S P with P = I except P_row = V diag(s) V^T
    (V orthogonal, s spanning `decades` decades): S' stays SPD, D'_row gets
    kappa ~ 10^(2 decades) kappa(D_row), and the preconditioned spectrum is
    unchanged (the preconditioner of Sec. 4.1 transforms with P)."""
    n = inst.n
    rng = np.random.default_rng(seed)
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Pm = V @ np.diag(np.logspace(0, -decades, n)) @ V.T
    D, O = inst.D.copy(), inst.O.copy()
    D[row] = Pm.T @ D[row] @ Pm
    D[row] = 0.5 * (D[row] + D[row].T)
    if row > 0:
        O[row - 1] = O[row - 1] @ Pm
    if row < inst.N - 1:
        O[row] = Pm.T @ O[row]
    from paper_2503_15269_gb300 import workloads as wl
    return wl.Instance(D=D, O=O, b=inst.b)
