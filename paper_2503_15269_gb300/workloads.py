"""Seeded synthetic instances of SPD block-tridiagonal systems S x = b.

This module only draws inputs: it holds none of the preconditioner or
solver arithmetic, so both the CUDA path and the CPU oracle can be fed from
it without sharing any of the method's code.

Matrix layout (Sec. 2.1, Eq. 1; 0-based here, the paper counts from 1):
    D : float64 [N, n, n]    diagonal blocks D_i (SPD, row-major)
    O : float64 [N-1, n, n]  super-diagonal blocks O_i = S[i, i+1];
                             S[i+1, i] = O_i^T
    b : float64 [N, n] or [N, n, nrhs]

Two families are generated:

* ``llt``  -- S = L L^T with L lower block-bidiagonal.  Diagonal blocks L_i
  are lower triangular with diagonal U[1, 2] and strict-lower entries of
  variance 0.1 * (6/n); sub-diagonal blocks M_i have entries of variance
  0.25 * (6/n).  At n = 6 this is exactly the published small case; the
  6/n factor keeps each row's norm fixed as n grows (without it the
  n = 48 case is numerically singular, kappa > 1e16 already at N = 16).
* ``ocp``  -- Schur complement S = C G^-1 C^T of an LQR problem with N knot
  points (Sec. 5 builds its test matrices this way): states x_0..x_{N-1},
  inputs u_0..u_{N-2}, dynamics x_{k+1} = A_k x_k + B_k u_k, x_0 fixed,
  Hessian G = blkdiag(Q_0, R_0, Q_1, ..., R_{N-2}, Q_{N-1}).  Then
      D_0     = Q_0^-1
      D_{k+1} = A_k Q_k^-1 A_k^T + B_k R_k^-1 B_k^T + Q_{k+1}^-1
      O_k     = -Q_k^-1 A_k^T
  with A_k = I + 0.05 N(0,1), B_k = 0.05 N(0,1) (n x m), Q_k = diag U[1,10],
  R_k = diag U[0.1, 1].

Seeds: instance k of workload c uses numpy PCG64 seeded with
1_000_003 * c + k; b is drawn after the matrix from the same stream.  The
(N, n) draws of the mixed batch come from a separate stream seeded with
(1_000_003 * c, 7).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

SEED_STRIDE = 1_000_003


def _rng(config: int, instance: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_STRIDE * config + instance))


@dataclasses.dataclass
class Instance:
    D: np.ndarray          # [N, n, n]
    O: np.ndarray          # [N-1, n, n]
    b: np.ndarray          # [N, n] or [N, n, nrhs]
    L: Optional[np.ndarray] = None   # llt family only: diagonal factors L_i
    M: Optional[np.ndarray] = None   # llt family only: sub-diagonal factors M_i

    @property
    def N(self) -> int:
        return self.D.shape[0]

    @property
    def n(self) -> int:
        return self.D.shape[1]


def llt_instance(rng: np.random.Generator, N: int, n: int, nrhs: int = 0) -> Instance:
    """Block-bidiagonal factor L, S = L L^T (see module docstring)."""
    s = 6.0 / n
    L = np.tril(rng.normal(0.0, np.sqrt(0.1 * s), (N, n, n)), -1)
    idx = np.arange(n)
    L[:, idx, idx] = rng.uniform(1.0, 2.0, (N, n))
    M = rng.normal(0.0, 0.5 * np.sqrt(s), (max(N - 1, 0), n, n))
    # S[i,i] = L_i L_i^T + M_{i-1} M_{i-1}^T ; S[i,i+1] = L_i M_i^T
    D = np.einsum("kij,klj->kil", L, L)
    if N > 1:
        D[1:] += np.einsum("kij,klj->kil", M, M)
    O = np.einsum("kij,klj->kil", L[:-1], M) if N > 1 else np.zeros((0, n, n))
    shape = (N, n) if nrhs == 0 else (N, n, nrhs)
    b = rng.standard_normal(shape)
    return Instance(D=D, O=O, b=b, L=L, M=M)


def ocp_instance(rng: np.random.Generator, N: int, n: int, m: int, nrhs: int = 0) -> Instance:
    """LQR Schur complement (see module docstring)."""
    A = np.eye(n) + 0.05 * rng.standard_normal((max(N - 1, 0), n, n))
    B = 0.05 * rng.standard_normal((max(N - 1, 0), n, m))
    Q = rng.uniform(1.0, 10.0, (N, n))
    R = rng.uniform(0.1, 1.0, (max(N - 1, 0), m))
    Qi = 1.0 / Q
    Ri = 1.0 / R
    D = np.zeros((N, n, n))
    O = np.zeros((max(N - 1, 0), n, n))
    D[0] = np.diag(Qi[0])
    for k in range(N - 1):
        AQ = A[k] * Qi[k][None, :]                       # A_k Q_k^-1
        D[k + 1] = AQ @ A[k].T + (B[k] * Ri[k][None, :]) @ B[k].T + np.diag(Qi[k + 1])
        O[k] = -(Qi[k][:, None] * A[k].T)                # -Q_k^-1 A_k^T
    shape = (N, n) if nrhs == 0 else (N, n, nrhs)
    b = rng.standard_normal(shape)
    return Instance(D=D, O=O, b=b)


# ---------------------------------------------------------------------------
# The five published workloads.
# ---------------------------------------------------------------------------

WORKLOADS = {
    0: "llt N=16 n=6, FP64, tol 1e-10",
    1: "ocp N=128 n=12 m=4, single instance, FP64 and mixed",
    2: "ocp batch of 1024, N~U{32..512}, n in {12,24,36}, m=n/3, mixed",
    3: "llt N=2048 n=48, 64 right-hand sides, mixed (tensor-core block products)",
    4: "ocp batch of 256, N=256 n=24 m=8, mixed, forward + adjoint",
}


def config0() -> Instance:
    return llt_instance(_rng(0, 0), 16, 6)


def config1() -> Instance:
    return ocp_instance(_rng(1, 0), 128, 12, 4)


def config2_shapes(count: int = 1024) -> List[tuple]:
    g = np.random.Generator(np.random.PCG64([SEED_STRIDE * 2, 7]))
    Ns = g.integers(32, 513, size=count)
    ns = g.choice(np.array([12, 24, 36]), size=count)
    return [(int(N), int(n)) for N, n in zip(Ns, ns)]


def config2(count: int = 1024, indices: Optional[List[int]] = None) -> List[Instance]:
    """The mixed batch; ``indices`` selects a subset (same draws as the full batch)."""
    shapes = config2_shapes(count)
    idx = range(count) if indices is None else indices
    return [ocp_instance(_rng(2, k), shapes[k][0], shapes[k][1], shapes[k][1] // 3) for k in idx]


def config3(N: int = 2048, n: int = 48, nrhs: int = 64) -> Instance:
    return llt_instance(_rng(3, 0), N, n, nrhs=nrhs)


def config4(count: int = 256, N: int = 256, n: int = 24, m: int = 8,
            indices: Optional[List[int]] = None) -> List[Instance]:
    idx = range(count) if indices is None else indices
    return [ocp_instance(_rng(4, k), N, n, m) for k in idx]


def small_llt(seed: int, N: int, n: int, nrhs: int = 0) -> Instance:
    """Extra small cases for tests (seed space disjoint from the workloads)."""
    return llt_instance(_rng(100 + seed, N * 1000 + n), N, n, nrhs=nrhs)


def small_ocp(seed: int, N: int, n: int, m: Optional[int] = None) -> Instance:
    return ocp_instance(_rng(200 + seed, N * 1000 + n), N, n, m if m is not None else max(1, n // 3))


@dataclasses.dataclass
class LQRData:
    """An LQR problem (Sec. 5 builds its matrices from such problems):
    A [N-1, n, n], Bm [N-1, n, m], Q [N, n, n], R [N-1, m, m] (dense SPD),
    q [N, n], r [N-1, m], c [N, n] (c_0 the initial state, c_{k+1} the
    affine term of the dynamics x_{k+1} = A_k x_k + B_k u_k + c_{k+1})."""
    A: np.ndarray
    Bm: np.ndarray
    Q: np.ndarray
    R: np.ndarray
    q: np.ndarray
    r: np.ndarray
    c: np.ndarray

    @property
    def N(self) -> int:
        return self.Q.shape[0]

    @property
    def n(self) -> int:
        return self.Q.shape[1]

    @property
    def m(self) -> int:
        return self.R.shape[1]


def lqr_data(rng: np.random.Generator, N: int, n: int, m: int) -> LQRData:
    """A_k = I + 0.05 N(0,1), B_k = 0.05 N(0,1) as in ocp_instance; dense SPD
    Q_k = diag U[1,10] + M M^T / n and R_k = diag U[0.1,1] + P P^T / m with
    M, P entries 0.3 N(0,1); q, r, c_0 ~ N(0,1), c_{k+1} ~ 0.1 N(0,1)."""
    A = np.eye(n) + 0.05 * rng.standard_normal((max(N - 1, 0), n, n))
    Bm = 0.05 * rng.standard_normal((max(N - 1, 0), n, m))
    Mq = 0.3 * rng.standard_normal((N, n, n))
    Q = np.stack([np.diag(rng.uniform(1.0, 10.0, n)) + Mq[k] @ Mq[k].T / n for k in range(N)])
    Pr = 0.3 * rng.standard_normal((max(N - 1, 0), m, m))
    R = (np.stack([np.diag(rng.uniform(0.1, 1.0, m)) + Pr[k] @ Pr[k].T / m for k in range(N - 1)])
         if N > 1 else np.zeros((0, m, m)))
    q = rng.standard_normal((N, n))
    r = rng.standard_normal((max(N - 1, 0), m))
    c = np.concatenate([rng.standard_normal((1, n)), 0.1 * rng.standard_normal((max(N - 1, 0), n))])
    return LQRData(A, Bm, Q, R, q, r, c)


def small_lqr(seed: int, N: int, n: int, m: int) -> LQRData:
    return lqr_data(_rng(300 + seed, N * 1000 + n), N, n, m)


# The experiment protocol of the numerical-results section (Sec. 5): five
# settings of the family, m = 1..4, 100 LQR matrices N = 30, n = 20 with 100
# right-hand sides each, PCG to ||S x - b||_2 < 1e-6.
PROTOCOL_SETTINGS = [("block Jacobi", 0.0, False), ("equal", 1.0 / 3.0, False), ("stairs only", 0.5, False),
                     ("optimal", 1.0, False), ("PolyCoeff", 1.0, True)]


def protocol_alpha(m: int, polycoeff: bool) -> List[float]:
    """Polynomial coefficients of a protocol setting: all ones, or for
    PolyCoeff alpha_{m-1} = 7 (the footnote's grid-search value)."""
    alpha = [1.0] * m
    if polycoeff and m > 1:
        alpha[-1] = 7.0
    return alpha


def protocol_batch(nmat: int = 100, nrhs: int = 100, N: int = 30, n: int = 20):
    """nmat LQR matrices, each repeated for nrhs right-hand sides drawn
    standard normal and scaled to unit norm (so the relative tolerance 1e-6 is
    the absolute exit rule); packed like pack_batch, instance k = (matrix
    k // nrhs, right-hand side k % nrhs)."""
    mats = [ocp_instance(_rng(5, k), N, n, max(1, n // 3)) for k in range(nmat)]
    B = nmat * nrhs
    D = np.repeat(np.stack([m.D for m in mats]), nrhs, axis=0).reshape(-1)
    O = np.repeat(np.stack([m.O for m in mats]), nrhs, axis=0).reshape(-1)
    g = np.random.Generator(np.random.PCG64([SEED_STRIDE * 5, 1]))
    b = g.standard_normal((B, N * n))
    b /= np.linalg.norm(b, axis=1, keepdims=True)
    Ns = np.full(B, N, dtype=np.int32)
    ns = np.full(B, n, dtype=np.int32)
    d_off = np.arange(B, dtype=np.int64) * N * n * n
    o_off = np.arange(B, dtype=np.int64) * (N - 1) * n * n
    v_off = np.arange(B, dtype=np.int64) * N * n
    return Ns, ns, d_off, o_off, v_off, D, O, b.reshape(-1)


def pack_batch(instances: List[Instance]):
    """Pack a batch back to back: returns (N[], n[], d_off[], o_off[], vec_off[], D, O, b).

    Offsets are element offsets.  Instance k's D occupies N_k*n_k*n_k doubles
    from d_off[k]; its O occupies (N_k-1)*n_k*n_k from o_off[k]; its b/x occupy
    N_k*n_k from vec_off[k].
    """
    Ns = np.array([i.N for i in instances], dtype=np.int32)
    ns = np.array([i.n for i in instances], dtype=np.int32)
    dsz = np.array([i.N * i.n * i.n for i in instances], dtype=np.int64)
    osz = np.array([max(i.N - 1, 0) * i.n * i.n for i in instances], dtype=np.int64)
    vsz = np.array([i.N * i.n for i in instances], dtype=np.int64)
    d_off = np.concatenate([[0], np.cumsum(dsz)[:-1]]).astype(np.int64)
    o_off = np.concatenate([[0], np.cumsum(osz)[:-1]]).astype(np.int64)
    v_off = np.concatenate([[0], np.cumsum(vsz)[:-1]]).astype(np.int64)
    D = np.concatenate([i.D.reshape(-1) for i in instances])
    O = np.concatenate([i.O.reshape(-1) for i in instances]) if osz.sum() else np.zeros(0)
    b = np.concatenate([i.b.reshape(-1) for i in instances])
    return Ns, ns, d_off, o_off, v_off, D, O, b
