"""CPU FP64 oracle for PCG on SPD block-tridiagonal systems with the
multi-splitting polynomial preconditioner of arXiv 2503.15269.

TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check in
__graft_entry__.py and bench.py's CPU-baseline leg may import this module.
It shares no code with the CUDA path and must never be used as a fallback
for it.

Everything is plain numpy/scipy in float64, written for readability rather
than speed: each function follows one passage of the paper and uses dense
library routines (cholesky, inv, triangular solves, matmul) as its steps.
Block indices are 0-based (the paper counts from 1).

Data layout (Sec. 2.1, Eq. 1):
    D : [N, n, n]    diagonal blocks D_i
    O : [N-1, n, n]  O_i = S[i, i+1];  S[i+1, i] = O_i^T
    vectors : [N, n] block vectors (or [N*n] flat)

Parity status: every function below is pinned by a test in
tests/test_oracle_*.py against something other than itself (dense library
solves/inverses/eigensolvers, the paper's closed forms, its spectral lemmas
and counts, finite differences, an independent second construction).
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Optional, Sequence

import numpy as np
import scipy.linalg as sla

# ---------------------------------------------------------------------------
# Status codes (same meaning as the C boundary's enum; defined here again on
# purpose -- the oracle shares no code with the library).
# ---------------------------------------------------------------------------
OK, NOT_SPD, NO_CONVERGENCE, BREAKDOWN, NONFINITE = 0, 3, 4, 5, 6


# ---------------------------------------------------------------------------
# Sec. 2.1, Eq. 1: the matrix class.
# ---------------------------------------------------------------------------
def assemble(D: np.ndarray, O: np.ndarray) -> np.ndarray:
    """Dense S from its blocks: S[i,i] = D_i, S[i,i+1] = O_i, S[i+1,i] = O_i^T."""
    N, n, _ = D.shape
    S = np.zeros((N * n, N * n))
    for i in range(N):
        S[i * n:(i + 1) * n, i * n:(i + 1) * n] = D[i]
    for i in range(N - 1):
        S[i * n:(i + 1) * n, (i + 1) * n:(i + 2) * n] = O[i]
        S[(i + 1) * n:(i + 2) * n, i * n:(i + 1) * n] = O[i].T
    return S


def spmv(D: np.ndarray, O: np.ndarray, x: np.ndarray) -> np.ndarray:
    """y = S x, block row by block row (Eq. 1):
    y_i = O_{i-1}^T x_{i-1} + D_i x_i + O_i x_{i+1}.  x: [N, n] or [N, n, k]."""
    N = D.shape[0]
    y = np.zeros_like(x)
    for i in range(N):
        y[i] = D[i] @ x[i]
        if i > 0:
            y[i] += O[i - 1].T @ x[i - 1]
        if i < N - 1:
            y[i] += O[i] @ x[i + 1]
    return y


# ---------------------------------------------------------------------------
# Sec. 4.3: the direct method, block Cholesky, O(N n^3) and sequential in N.
# This is the plain definition of the result x = S^-1 b.
# ---------------------------------------------------------------------------
def block_cholesky(D: np.ndarray, O: np.ndarray):
    """S = L L^T with L lower block-bidiagonal: L[i,i] = C_i (lower
    triangular), L[i+1,i] = F_i.
        C_0 C_0^T = D_0
        F_i = O_i^T C_i^-T
        C_{i+1} C_{i+1}^T = D_{i+1} - F_i F_i^T
    Returns (C, F, status, failing_block)."""
    N, n, _ = D.shape
    C = np.zeros_like(D)
    F = np.zeros((max(N - 1, 0), n, n))
    U = D[0].copy()
    for i in range(N):
        try:
            C[i] = np.linalg.cholesky(U)
        except np.linalg.LinAlgError:
            return C, F, NOT_SPD, i
        if i < N - 1:
            # F_i = O_i^T C_i^-T  <=>  C_i F_i^T = O_i
            F[i] = sla.solve_triangular(C[i], O[i], lower=True).T
            U = D[i + 1] - F[i] @ F[i].T
    return C, F, OK, -1


def direct_solve(D: np.ndarray, O: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x = S^-1 b by block forward/back substitution on the block Cholesky
    factor (Sec. 4.3).  b: [N, n] or [N, n, k]."""
    C, F, st, blk = block_cholesky(D, O)
    if st != OK:
        raise np.linalg.LinAlgError(f"block {blk} not positive definite")
    N = D.shape[0]
    y = np.zeros_like(b)
    for i in range(N):
        rhs = b[i] - (F[i - 1] @ y[i - 1] if i > 0 else 0.0)
        y[i] = sla.solve_triangular(C[i], rhs, lower=True)
    x = np.zeros_like(b)
    for i in reversed(range(N)):
        rhs = y[i] - (F[i].T @ x[i + 1] if i < N - 1 else 0.0)
        x[i] = sla.solve_triangular(C[i], rhs, lower=True, trans="T")
    return x


# ---------------------------------------------------------------------------
# Sec. 2.3: the diagonal splitting and the two stair splittings, dense.
# Used by the spectral and closed-form checks on small inputs.
# ---------------------------------------------------------------------------
def splittings(D: np.ndarray, O: np.ndarray):
    """Dense (B_d, C_d, B_l, C_l, B_r, C_r) with A = B - C for each.

    B_d = blkdiag(D_i).  B_l keeps whole the block rows that are even in the
    paper's 1-based count (odd 0-based index) and keeps only D_i on the
    others; B_r does the opposite (Eq. for the stair splittings, drawn there
    for N = 3)."""
    N, n, _ = D.shape
    A = assemble(D, O)
    Bd = np.zeros_like(A)
    for i in range(N):
        Bd[i * n:(i + 1) * n, i * n:(i + 1) * n] = D[i]
    Bl = Bd.copy()
    Br = Bd.copy()
    for i in range(N):
        rows = slice(i * n, (i + 1) * n)
        target = Bl if i % 2 == 1 else Br
        target[rows, :] = A[rows, :]
    return Bd, Bd - A, Bl, Bl - A, Br, Br - A


def GH_dense(D: np.ndarray, O: np.ndarray, a: float):
    """(G_ab, H_ab) straight from the multi-splitting definition (Sec. 3.1):
        G_ab = a (B_l^-1 + B_r^-1) + b B_d^-1
        H_ab = a (B_l^-1 C_l + B_r^-1 C_r) + b B_d^-1 C_d,   b = 1 - 2a."""
    Bd, Cd, Bl, Cl, Br, Cr = splittings(D, O)
    b = 1.0 - 2.0 * a
    Bli, Bri, Bdi = np.linalg.inv(Bl), np.linalg.inv(Br), np.linalg.inv(Bd)
    G = a * (Bli + Bri) + b * Bdi
    H = a * (Bli @ Cl + Bri @ Cr) + b * (Bdi @ Cd)
    return G, H


# ---------------------------------------------------------------------------
# Sec. 4.1: closed-form blocks of (G_opt, H_opt) at a = 1, b = -1.
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class OptBlocks:
    Dinv: np.ndarray   # [N, n, n]     D_i^-1                 (G diagonal)
    E: np.ndarray      # [N-1, n, n]   E_i = D_i^-1 O_i D_{i+1}^-1; G[i,i+1] = -E_i, G[i+1,i] = -E_i^T
    Hd: np.ndarray     # [N, n, n]     H[i,i]   = E_{i-1}^T O_{i-1} + E_i O_i^T
    Hu: np.ndarray     # [N-2, n, n]   H[i,i+2] = E_i O_{i+1}
    Hl: np.ndarray     # [N-2, n, n]   H[i+2,i] = E_{i+1}^T O_i^T


def opt_blocks(D: np.ndarray, O: np.ndarray) -> OptBlocks:
    """E_i := D_i^-1 O_i D_{i+1}^-1 and the block pattern of G_opt
    (tridiagonal) and H_opt (pentadiagonal with zero +-1 blocks), Sec. 4.1."""
    N, n, _ = D.shape
    Dinv = np.stack([np.linalg.inv(D[i]) for i in range(N)])
    E = np.stack([Dinv[i] @ O[i] @ Dinv[i + 1] for i in range(N - 1)]) if N > 1 else np.zeros((0, n, n))
    Hd = np.zeros_like(D)
    for i in range(N):
        if i > 0:
            Hd[i] += E[i - 1].T @ O[i - 1]
        if i < N - 1:
            Hd[i] += E[i] @ O[i].T
    Hu = np.stack([E[i] @ O[i + 1] for i in range(N - 2)]) if N > 2 else np.zeros((0, n, n))
    Hl = np.stack([E[i + 1].T @ O[i].T for i in range(N - 2)]) if N > 2 else np.zeros((0, n, n))
    return OptBlocks(Dinv, E, Hd, Hu, Hl)


def apply_G_opt(B: OptBlocks, r: np.ndarray) -> np.ndarray:
    """y = G_opt r: y_i = D_i^-1 r_i - E_i r_{i+1} - E_{i-1}^T r_{i-1}."""
    N = B.Dinv.shape[0]
    y = np.zeros_like(r)
    for i in range(N):
        y[i] = B.Dinv[i] @ r[i]
        if i < N - 1:
            y[i] -= B.E[i] @ r[i + 1]
        if i > 0:
            y[i] -= B.E[i - 1].T @ r[i - 1]
    return y


def apply_H_opt(B: OptBlocks, y: np.ndarray) -> np.ndarray:
    """w = H_opt y: w_i = Hd_i y_i + Hu_i y_{i+2} + Hl_{i-2} y_{i-2}."""
    N = B.Dinv.shape[0]
    w = np.zeros_like(y)
    for i in range(N):
        w[i] = B.Hd[i] @ y[i]
        if i + 2 < N:
            w[i] += B.Hu[i] @ y[i + 2]
        if i - 2 >= 0:
            w[i] += B.Hl[i - 2] @ y[i - 2]
    return w


def apply_opt(B: OptBlocks, r: np.ndarray, alpha: Sequence[float]) -> np.ndarray:
    """z = (alpha_0 I + alpha_1 H + ... + alpha_{m-1} H^{m-1}) G r with
    alpha_0 = 1 (Eq. with polynomial coefficients, Sec. 3.5), computed as
    the paper prescribes in Sec. 4.2: y_0 = G r, y_j = H y_{j-1}."""
    y = apply_G_opt(B, r)
    z = alpha[0] * y
    for a_j in alpha[1:]:
        y = apply_H_opt(B, y)
        z = z + a_j * y
    return z


# ---------------------------------------------------------------------------
# The general member (a, 1-2a) of the family, in block form.  The paper
# omits these formulas (Sec. 4.1 says they follow like the optimal case);
# the reading used here is
#     G_ab = B_d^-1 + a B_d^-1 C_d B_d^-1
#     H_ab = (1 - a) H_J + a H_J^2,   H_J = B_d^-1 C_d,
# which the tests check densely against GH_dense for several a.
# ---------------------------------------------------------------------------
def apply_HJ(Dinv: np.ndarray, O: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Block-Jacobi iteration matrix H_J = B_d^-1 C_d applied to y:
    (H_J y)_i = -D_i^-1 (O_{i-1}^T y_{i-1} + O_i y_{i+1})."""
    N = Dinv.shape[0]
    t = np.zeros_like(y)
    for i in range(N):
        if i > 0:
            t[i] += O[i - 1].T @ y[i - 1]
        if i < N - 1:
            t[i] += O[i] @ y[i + 1]
    return -np.einsum("kij,kj...->ki...", Dinv, t)


def apply_family(D: np.ndarray, O: np.ndarray, r: np.ndarray, a: float,
                 alpha: Sequence[float]) -> np.ndarray:
    """z = sum_j alpha_j H_ab^j G_ab r for any a in [0, 1]."""
    N = D.shape[0]
    Dinv = np.stack([np.linalg.inv(D[i]) for i in range(N)])
    u = np.einsum("kij,kj...->ki...", Dinv, r)                 # B_d^-1 r
    y = u + a * apply_HJ(Dinv, O, u)                            # G_ab r
    z = alpha[0] * y
    for a_j in alpha[1:]:
        hy = apply_HJ(Dinv, O, y)
        y = (1.0 - a) * hy + a * apply_HJ(Dinv, O, hy)          # H_ab y
        z = z + a_j * y
    return z


def apply_jacobi_sweeps(D: np.ndarray, O: np.ndarray, r: np.ndarray, m: int) -> np.ndarray:
    """Footnote to Thm. 3.2: _{1,-1}M_m^-1 = _{0,1}M_{2m}^-1, i.e. 2m
    block-Jacobi sweeps z <- B_d^-1 (r + C_d z) from z = 0.  A second,
    independent construction of the optimal preconditioner (alpha = 1)."""
    N = D.shape[0]
    z = np.zeros_like(r)
    for _ in range(2 * m):
        t = r.copy()                      # r + C_d z = r - offdiag(S) z
        for i in range(N):
            if i > 0:
                t[i] -= O[i - 1].T @ z[i - 1]
            if i < N - 1:
                t[i] -= O[i] @ z[i + 1]
        z = np.stack([np.linalg.solve(D[i], t[i]) for i in range(N)])
    return z


# ---------------------------------------------------------------------------
# PCG (the paper cites the textbook method, Nocedal-Wright; it prints none).
# Stopping rule: ||r_k||_2 <= tol * ||b||_2 on the recursive residual.
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class PCGResult:
    x: np.ndarray
    iters: int
    status: int
    res_history: list
    alphas: list
    betas: list


def pcg(D: np.ndarray, O: np.ndarray, b: np.ndarray, minv: Callable[[np.ndarray], np.ndarray],
        tol: float, maxit: int, x0: Optional[np.ndarray] = None) -> PCGResult:
    """Textbook preconditioned CG; iters counts products S p."""
    x = np.zeros_like(b) if x0 is None else x0.astype(np.float64).copy()
    r = b - spmv(D, O, x) if x0 is not None else b.copy()
    nb = np.linalg.norm(b)
    hist = [np.linalg.norm(r)]
    if not np.all(np.isfinite(b)) or not np.all(np.isfinite(r)):
        return PCGResult(x, 0, NONFINITE, hist, [], [])
    if nb == 0.0:
        return PCGResult(np.zeros_like(b), 0, OK, hist, [], [])
    if hist[0] <= tol * nb:
        return PCGResult(x, 0, OK, hist, [], [])
    z = minv(r)
    p = z.copy()
    rho = float(np.vdot(r, z))
    alphas, betas = [], []
    for k in range(1, maxit + 1):
        q = spmv(D, O, p)
        pq = float(np.vdot(p, q))
        if not (pq > 0.0) or not np.isfinite(pq):
            return PCGResult(x, k - 1, BREAKDOWN if np.isfinite(pq) else NONFINITE, hist, alphas, betas)
        al = rho / pq
        x = x + al * p
        r = r - al * q
        alphas.append(al)
        nr = np.linalg.norm(r)
        hist.append(nr)
        if not np.isfinite(nr):
            return PCGResult(x, k, NONFINITE, hist, alphas, betas)
        if nr <= tol * nb:
            return PCGResult(x, k, OK, hist, alphas, betas)
        z = minv(r)
        rho_new = float(np.vdot(r, z))
        be = rho_new / rho
        betas.append(be)
        p = z + be * p
        rho = rho_new
    return PCGResult(x, maxit, NO_CONVERGENCE, hist, alphas, betas)


def pcg_opt(D: np.ndarray, O: np.ndarray, b: np.ndarray, alpha: Sequence[float], tol: float,
            maxit: int, x0: Optional[np.ndarray] = None) -> PCGResult:
    """PCG with the optimal-parameter preconditioner (a = 1, b = -1) and
    coefficients alpha (alpha[0] = 1); blocks from the Sec. 4.1 closed form."""
    B = opt_blocks(D, O)
    return pcg(D, O, b, lambda r: apply_opt(B, r, alpha), tol, maxit, x0)


def lanczos_cond(alphas: Sequence[float], betas: Sequence[float]) -> float:
    """Condition-number estimate of M^-1 S from the CG coefficients: the
    Lanczos tridiagonal has diagonal 1/a_k + b_{k-1}/a_{k-1} and off-diagonal
    sqrt(b_k)/a_k (textbook relation); ratio of its extreme eigenvalues."""
    k = len(alphas)
    if k == 0:
        return 1.0
    d = np.array([1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0) for j in range(k)])
    e = np.array([np.sqrt(betas[j]) / alphas[j] for j in range(min(k - 1, len(betas)))])
    ev = sla.eigh_tridiagonal(d, e, eigvals_only=True)
    return float(ev[-1] / ev[0])


# ---------------------------------------------------------------------------
# Counts printed by the paper.
# ---------------------------------------------------------------------------
def d_Nna(N: int, n: int, a: float) -> int:
    """Distinct eigenvalues of _{ab}M_m^-1 A (Thm. 3.2, Eq. for d_Nna)."""
    if a == 1.0:
        return (N // 2) * n if N % 2 == 0 else (N // 2) * n + 1
    return N * n if N % 2 == 0 else 2 * (N // 2) * n + 1


def g_a(m: int, a: float) -> int:
    """Block gemvs per PCG iteration (Sec. 4.2)."""
    if a == 0.0:
        return 2 * m + 2
    if a == 1.0:
        return 3 * m + 3
    return 5 * m + 1


def f_a(lam: np.ndarray, a: float, sign: int) -> np.ndarray:
    """f_{a+-}(lambda) = a lambda +- (1 - a) sqrt(lambda) (Sec. 3.2)."""
    return a * lam + sign * (1.0 - a) * np.sqrt(lam)


# ---------------------------------------------------------------------------
# Adjoint of x = S^-1 b with respect to b and the blocks.
# ---------------------------------------------------------------------------
def adjoint(D: np.ndarray, O: np.ndarray, x: np.ndarray, gx: np.ndarray):
    """Given x = S^-1 b and dL/dx = gx: g = S^-1 gx (S symmetric),
    dL/db = g, dL/dD_i = -g_i x_i^T, dL/dO_i = -(g_i x_{i+1}^T + x_i g_{i+1}^T),
    the last because O_i sits at S[i,i+1] and O_i^T at S[i+1,i]."""
    g = direct_solve(D, O, gx)
    N = D.shape[0]
    gD = -np.einsum("ki,kj->kij", g, x)
    gO = np.zeros((max(N - 1, 0),) + D.shape[1:])
    for i in range(N - 1):
        gO[i] = -(np.outer(g[i], x[i + 1]) + np.outer(x[i], g[i + 1]))
    return g, gD, gO


# ---------------------------------------------------------------------------
# Sec. 5: the test matrices are Schur complements of LQR KKT systems (the
# construction is deferred to the cited GPU QP solver and not printed).  The
# reading: the equality-constrained QP over z = (x_0, u_0, x_1, ..., u_{N-2},
# x_{N-1}),
#     min 1/2 z^T G z + g^T z   s.t.  C z = c,
#     G = blkdiag(Q_0, R_0, Q_1, ..., R_{N-2}, Q_{N-1}),  g = (q_0, r_0, ..., q_{N-1}),
# with block rows of C: x_0 = c_0 (initial state) and
# x_{k+1} - A_k x_k - B_k u_k = c_{k+1} (dynamics with an affine term).
# Eliminating z from the KKT system [G C^T; C 0][z; lam] = [-g; c]:
#     S lam = gamma,  S = C G^-1 C^T,  gamma = -(c + C G^-1 g),
#     z = -G^-1 (g + C^T lam).
# Shapes: A [N-1, n, n], Bm [N-1, n, m], Q [N, n, n], R [N-1, m, m],
# q [N, n], r [N-1, m], c [N, n]; lam [N, n]; x [N, n], u [N-1, m].
# ---------------------------------------------------------------------------
def lqr_dense(A, Bm, Q, R, q, r, c):
    """Dense (G, g, C, c) of the QP, z ordered as above."""
    N, n = Q.shape[0], Q.shape[1]
    m = R.shape[1] if N > 1 else 0
    nz = N * n + (N - 1) * m
    xc = lambda k: k * (n + m)          # column of x_k in z
    uc = lambda k: k * (n + m) + n      # column of u_k in z
    G = np.zeros((nz, nz))
    g = np.zeros(nz)
    C = np.zeros((N * n, nz))
    for k in range(N):
        G[xc(k):xc(k) + n, xc(k):xc(k) + n] = Q[k]
        g[xc(k):xc(k) + n] = q[k]
        C[k * n:(k + 1) * n, xc(k):xc(k) + n] = np.eye(n)
        if k < N - 1:
            G[uc(k):uc(k) + m, uc(k):uc(k) + m] = R[k]
            g[uc(k):uc(k) + m] = r[k]
            C[(k + 1) * n:(k + 2) * n, xc(k):xc(k) + n] = -A[k]
            C[(k + 1) * n:(k + 2) * n, uc(k):uc(k) + m] = -Bm[k]
    return G, g, C, np.asarray(c, dtype=np.float64).reshape(-1)


def lqr_schur(A, Bm, Q, R, q, r, c):
    """(D, O, gamma): the blocks of S = C G^-1 C^T and gamma = -(c + C G^-1 g),
    formed densely and cut into block rows."""
    N, n = Q.shape[0], Q.shape[1]
    G, g, C, cv = lqr_dense(A, Bm, Q, R, q, r, c)
    Gi_Ct = np.linalg.solve(G, C.T)
    S = C @ Gi_Ct
    gamma = -(cv + C @ np.linalg.solve(G, g))
    D = np.stack([S[i * n:(i + 1) * n, i * n:(i + 1) * n] for i in range(N)])
    O = (np.stack([S[i * n:(i + 1) * n, (i + 1) * n:(i + 2) * n] for i in range(N - 1)])
         if N > 1 else np.zeros((0, n, n)))
    return D, O, gamma.reshape(N, n)


def lqr_recover(A, Bm, Q, R, q, r, lam):
    """z = -G^-1 (g + C^T lam), returned as (x [N, n], u [N-1, m])."""
    N, n = Q.shape[0], Q.shape[1]
    m = R.shape[1] if N > 1 else 0
    G, g, C, _ = lqr_dense(A, Bm, Q, R, q, r, np.zeros((N, n)))
    z = -np.linalg.solve(G, g + C.T @ np.asarray(lam, dtype=np.float64).reshape(-1))
    x = np.stack([z[k * (n + m):k * (n + m) + n] for k in range(N)])
    u = (np.stack([z[k * (n + m) + n:(k + 1) * (n + m)] for k in range(N - 1)])
         if N > 1 else np.zeros((0, m)))
    return x, u


# ---------------------------------------------------------------------------
# Polynomial coefficients beyond grid search (the paper's stated future work,
# Sec. 6).  At a = 1 the preconditioned matrix M^-1 S has the eigenvalues
# phi(h) = q(h) (1 - h), q(h) = sum_j alpha_j h^j, over the eigenvalues h of
# H_opt in [0, rho] (Sec. 3.5).  The q of degree m-1 that makes phi closest to
# a constant on [0, rho] -- the smallest max |1 - c phi(h)| -- comes from the
# shifted Chebyshev polynomial T_m (the classic minimax property):
#     p(h) = T_m((2h - rho)/rho) / T_m((2 - rho)/rho),   p(1) = 1,
#     q(h) = (1 - p(h)) / (1 - h)   (exact division, 1 - p vanishes at 1),
# normalised to alpha_0 = 1 (scaling M^-1 does not change PCG's iterates).
# ---------------------------------------------------------------------------
def chebyshev_alpha(m: int, rho: float) -> np.ndarray:
    """alpha (length m, alpha_0 = 1) of the Chebyshev choice for rho(H_opt) <= rho."""
    P = np.polynomial.polynomial
    # T_0 = 1, T_1 = x, T_{k+1} = 2 x T_k - T_{k-1}, in the variable
    # x = (2h - rho)/rho, as power-basis coefficient arrays in h
    x = np.array([-1.0, 2.0 / rho])
    t_prev, t = np.array([1.0]), x.copy()
    if m == 0:
        t = t_prev
    for _ in range(m - 1):
        t_prev, t = t, P.polysub(2.0 * P.polymul(x, t), t_prev)
    p = t / P.polyval(1.0, t)                       # p(1) = 1
    one_minus_p = P.polysub(np.array([1.0]), p)
    q, rem = P.polydiv(one_minus_p, np.array([1.0, -1.0]))
    assert np.allclose(rem, 0.0, atol=1e-9 * np.abs(one_minus_p).max())
    q = np.asarray(q, dtype=np.float64)
    q = np.concatenate([q, np.zeros(max(0, m - q.size))])[:m]
    return q / q[0]


def power_rho(D: np.ndarray, O: np.ndarray, iters: int) -> float:
    """Estimate of the spectral radius of H_opt by power iteration, using
    M^-1 S = I - H_opt for the optimum at m = 1 (Sec. 3.5): from
    v_i = 1 + sin(i)/10 (normalised), v <- h / ||h|| with h = v - G_opt S v;
    returns ||h|| of the last step (H_opt is not symmetric: the ratio can
    end slightly above rho)."""
    B = opt_blocks(D, O)
    N, n = D.shape[0], D.shape[1]
    v = (1.0 + 0.1 * np.sin(np.arange(N * n, dtype=np.float64))).reshape(N, n)
    v = v / np.linalg.norm(v)
    nh = 0.0
    for _ in range(iters):
        h = v - apply_G_opt(B, spmv(D, O, v))
        nh = float(np.linalg.norm(h))
        v = h / nh
    return nh


def ritz_rho(D: np.ndarray, O: np.ndarray, b: np.ndarray, iters: int) -> float:
    """rho(H_opt) estimated from Ritz values: `iters` iterations of textbook
    PCG with M^-1 = G_opt (m = 1, where M^-1 S = I - H_opt, Sec. 3.5); the
    CG scalars give the Lanczos tridiagonal T of the preconditioned operator
    (T_00 = 1/a_0, T_jj = 1/a_j + b_{j-1}/a_{j-1}, T_j,j-1 = sqrt(b_{j-1})/a_{j-1});
    returns 1 - lambda_min(T)."""
    B = opt_blocks(D, O)
    res = pcg(D, O, b, lambda r: apply_G_opt(B, r), 0.0, iters)
    a, be = res.alphas, res.betas
    K = min(len(a), len(be) + 1)
    T = np.zeros((K, K))
    for j in range(K):
        T[j, j] = 1.0 / a[j] + (be[j - 1] / a[j - 1] if j > 0 else 0.0)
        if j > 0:
            T[j, j - 1] = T[j - 1, j] = np.sqrt(be[j - 1]) / a[j - 1]
    return 1.0 - float(np.linalg.eigvalsh(T).min())
