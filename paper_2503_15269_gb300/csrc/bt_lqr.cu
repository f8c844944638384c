// LQR problems -> the block-tridiagonal Schur complement the solver takes,
// and the dual-to-primal recovery after the solve (the construction of the
// test matrices of Sec. 5: an LQR problem as an equality-constrained QP, its
// KKT system, and the Schur complement with respect to the Hessian).
//
// QP over z = (x_0, u_0, x_1, ..., u_{N-2}, x_{N-1}):
//     min 1/2 z^T G z + g^T z   s.t.  C z = c,
//     G = blkdiag(Q_0, R_0, ..., R_{N-2}, Q_{N-1}),  g = (q_0, r_0, ..., q_{N-1}),
//     C: x_0 = c_0,  x_{k+1} - A_k x_k - B_k u_k = c_{k+1}.
// Eliminating z from [G C^T; C 0][z; lam] = [-g; c]:
//     S lam = gamma,  S = C G^-1 C^T,  gamma = -(c + C G^-1 g),
//     z = -G^-1 (g + C^T lam),
// and in blocks, with P_k = Q_k^-1 A_k^T and w_k = Q_k^-1 q_k:
//     D_0 = Q_0^-1,  D_k = Q_k^-1 + A_{k-1} P_{k-1} + B_{k-1} R_{k-1}^-1 B_{k-1}^T,
//     O_k = -P_k,
//     gamma_k = -(c_k + w_k - A_{k-1} w_{k-1} - B_{k-1} R_{k-1}^-1 r_{k-1}),
//     x_k = -Q_k^-1 (q_k + lam_k - A_k^T lam_{k+1}),  u_k = -R_k^-1 (r_k - B_k^T lam_{k+1}).
//
// The blocks feed the float64 residual of the solver, so they are formed to
// float64 accuracy: the formation in double-float pairs on the float32 pipe
// (float64 issues at ~2 FMA per clock per SM on GB300, 1/64 of float32),
// the recovery in float64.  One CTA walks a segment of consecutive block
// rows of one instance and carries row k-1's contribution to D_k and gamma_k
// in shared memory from row to row.
#include <algorithm>
#include <vector>

#include "../../include/bt.h"
#include "bt_common.cuh"
#include "bt_dd.cuh"

namespace bt {

constexpr int kLqrThreads = 128;
constexpr int kLqrSeg = 16;  // block rows per CTA segment
constexpr int kLqrMax = 48;  // largest n and m (shared-memory budget)
static_assert(kLqrThreads >= kLqrMax, "one thread per row of a block column");

struct LqrDesc {
  int N, n, m, pad;
  long long oA, oB, oQ, oR, ov, ou;  // element offsets: A/O, Bm, Q/D, R, n-vectors, m-vectors
  long long ot;                      // first task of k_lqr_winv (sum over earlier problems of 2 N - 1)
  long long okn;                     // first knot (sum over earlier problems of N)
};
struct LqrSeg {
  int inst, a, b, pad;
};

struct LqrParams {
  const LqrDesc* desc;
  const LqrSeg* segs;
  const double *A, *Bm, *Q, *R, *q, *r, *c, *lam;
  double *D, *O, *gamma, *x, *u;
  dd *WQ, *WR;  // formation scratch: W = L^-1 of every Q_k, R_k (at the offsets of Q, R)
  // optional: a mixed handle's block arrays, written by the formation
  // (column-major slots at the handle's offsets) -- null when not attached
  const InstDesc* hinst;
  double *hD64, *hO64;
  float *hD32, *hO32, *hDinv32;
  unsigned long long* fail_key;  // min over (inst << 32 | 2 * row + (R ? 1 : 0)) of refused blocks
};

// ---- CTA-wide float64 helpers on row-major blocks in shared memory ---------

// Cholesky M = L L^T in place (lower triangle); false if a pivot is not
// positive.  Right-looking, two barriers per column: column j is scaled by
// the threads of its rows (each forms 1/L_jj itself), then the trailing
// triangle takes one FMA per element from the whole CTA.  Float64 issues at
// about 2 FMA per clock per SM here, so the multiplications stay out of the
// O(n^2)-per-step loops and every step spreads over all warps.
__device__ bool chol(double* M, int n, double* rinv) {
  for (int j = 0; j < n; ++j) {
    __syncthreads();
    const double piv = M[j * n + j];
    if (!(piv > 0.0) || !isfinite(piv)) return false;  // the same answer on every thread
    if (threadIdx.x < n - j) {
      const double ri = rsqrt(piv);
      const int r = j + threadIdx.x;
      M[r * n + j] = (r == j) ? piv * ri : M[r * n + j] * ri;
      if (threadIdx.x == 0) rinv[j] = ri;  // 1 / L_jj
    }
    __syncthreads();
    const int w = n - j - 1;
    for (int t = threadIdx.x; t < w * (w + 1) / 2; t += blockDim.x) {
      int rq = __float2int_rz((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);  // t -> (rq, cq), cq <= rq
      if ((rq + 1) * (rq + 2) / 2 <= t) ++rq;
      if (rq * (rq + 1) / 2 > t) --rq;
      const int r = j + 1 + rq, cc = j + 1 + (t - rq * (rq + 1) / 2);
      M[r * n + cc] = fma(-M[r * n + j], M[cc * n + j], M[r * n + cc]);
    }
  }
  __syncthreads();
  return true;
}

__device__ void load(double* dst, const double* src, int cnt) {
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) dst[t] = src[t];
}

__device__ void refuse(const LqrParams& P, int inst, int row, int isR) {
  if (threadIdx.x == 0)
    atomicMin(P.fail_key, ((unsigned long long)inst << 32) | (unsigned)(2 * row + isR));
}

// ---- formation ---------------------------------------------------------------
// Double-float (bt_dd.cuh) throughout the O(n^3) work: float64 runs at 1/64
// of the float32 rate here, and a pair of float32 numbers with error-free
// products and sums carries about 48 significand bits.  The inputs are split
// into pairs on load and the blocks rounded once to float64 on the store.
//
// Two kernels.  k_lqr_winv inverts the Cholesky factor of every Q_k and R_k,
// one warp per matrix with no CTA barrier (the column-serial part of a
// Cholesky is latency, so many independent matrices per SM hide it):
//   Q_k = L L^T,  W = L^-1 (so Q_k^-1 = W^T W), likewise W_R for R_k,
// into a scratch array of pairs.  k_lqr_schur then forms, per block row k,
//   Y = W A_k^T,  O_k = -W^T Y (= -Q_k^-1 A_k^T),  t = W q_k,  w_k = W^T t,
//   D_k = W^T W + C_{k-1},  gamma_k = -(c_k + w_k - g_{k-1}),
// and for the next row, with V = W_R B_k^T and s = W_R r_k,
//   C_k = Y^T Y + V^T V   (= A_k Q_k^-1 A_k^T + B_k R_k^-1 B_k^T),
//   g_k = Y^T t + V^T s   (= A_k w_k + B_k R_k^-1 r_k),
// from products only (every phase parallel over output elements).  With a
// mixed handle attached it writes D and O in the handle's layout (float64
// and float32 column-major slots) instead of, or besides, the caller's.

constexpr int kWinvWarps = 4;

// One warp: M (col-major pairs, n x n, element (i, j) at j n + i) <- the
// float64 row-major block src; Cholesky factor L in the lower triangle by
// columns (left-looking: lane = row, rows lane and lane + 32), rv[j] =
// 1 / L_jj; then W = L^-1 by columns (lane = column), W(i, c) for i > c kept
// in the upper triangle at index i n + c.  False (on every lane) if a pivot
// is not positive.
__device__ bool dd_warp_chol_inv(dd* M, dd* rv, const double* src, int n, int lane) {
  constexpr unsigned FULL = 0xffffffffu;
  for (int t = lane; t < n * n; t += 32) {
    const int i = t / n, j = t - i * n;
    M[j * n + i] = dd_from(src[t]);
  }
  __syncwarp();
  for (int j = 0; j < n; ++j) {
    dd dv[2] = {dd_make(0.f, 0.f), dd_make(0.f, 0.f)};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = lane + 32 * h;
      if (i < n && i >= j) {  // d_i = M(i, j) - sum_{p<j} L(i, p) L(j, p), two interleaved sums
        DDAcc a0, a1;
        a0.init(M[j * n + i]);
        a1.init0();
        int p = 0;
        for (; p + 1 < j; p += 2) {
          a0.fms(M[p * n + i], M[p * n + j]);
          a1.fms(M[(p + 1) * n + i], M[(p + 1) * n + j]);
        }
        if (p < j) a0.fms(M[p * n + i], M[p * n + j]);
        dv[h] = dd_add(a0.value(), a1.value());
      }
    }
    const dd own = (j < 32) ? dv[0] : dv[1];
    const dd piv = dd_make(__shfl_sync(FULL, own.h, j & 31), __shfl_sync(FULL, own.l, j & 31));
    if (!(piv.h > 0.f) || !isfinite(piv.h)) return false;
    const dd s = dd_sqrt(piv);
    const dd r = dd_rcp(s);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = lane + 32 * h;
      if (i < n && i > j) M[j * n + i] = dd_mul(dv[h], r);
    }
    if (lane == (j & 31)) {
      M[j * n + j] = s;
      rv[j] = r;
    }
    __syncwarp();
  }
  // W(i, c) = -(1 / L_ii) sum_{p=c}^{i-1} L(i, p) W(p, c), W(c, c) = 1 / L_cc;
  // a lane reads only its own column of W and the (read-only) lower triangle
  for (int i = 1; i < n; ++i) {
    const dd ri = rv[i];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = lane + 32 * h;
      if (c < i) {
        DDAcc a0, a1;
        a0.init0();
        a1.init0();
        a0.fma(M[c * n + i], rv[c]);
        int p = c + 1;
        for (; p + 1 < i; p += 2) {
          a0.fma(M[p * n + i], M[p * n + c]);
          a1.fma(M[(p + 1) * n + i], M[(p + 1) * n + c]);
        }
        if (p < i) a0.fma(M[p * n + i], M[p * n + c]);
        M[i * n + c] = dd_neg(dd_mul(dd_add(a0.value(), a1.value()), ri));
      }
    }
  }
  __syncwarp();
  return true;
}

// Every Q_k and R_k of the batch: task t of instance k (desc[k].ot <= t <
// desc[k+1].ot) is Q_{t - ot} for t - ot < N, else R_{t - ot - N}.  W is
// stored row-major (lower triangle, zeros above) at the element offset of
// its Q or R block.
__global__ void __launch_bounds__(kWinvWarps * 32) k_lqr_winv(const __grid_constant__ LqrParams P, long long ntask,
                                                               int B, int stride) {
  extern __shared__ __align__(16) double lsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long task = (long long)blockIdx.x * kWinvWarps + warp;
  if (task >= ntask) return;
  int lo = 0, hi = B - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P.desc[mid].ot <= task) lo = mid;
    else hi = mid - 1;
  }
  const LqrDesc d = P.desc[lo];
  const long long rel = task - d.ot;
  const bool isR = rel >= d.N;
  const int row = (int)(isR ? rel - d.N : rel);
  const int n = isR ? d.m : d.n;
  const long long off = isR ? d.oR + (long long)row * n * n : d.oQ + (long long)row * n * n;
  dd* M = reinterpret_cast<dd*>(lsm) + (size_t)warp * stride;
  dd* rv = M + n * n;
  if (!dd_warp_chol_inv(M, rv, (isR ? P.R : P.Q) + off, n, lane)) {
    if (lane == 0) atomicMin(P.fail_key, ((unsigned long long)lo << 32) | (unsigned)(2 * row + (isR ? 1 : 0)));
    return;
  }
  dd* dst = (isR ? P.WR : P.WQ) + off;
  for (int t = lane; t < n * n; t += 32) {
    const int i = t / n, c = t - i * n;
    dst[t] = (i > c) ? M[t] : (i == c ? rv[i] : dd_make(0.f, 0.f));
  }
}

// CTA-wide helpers of k_lqr_schur: every thread calls them; each ends with a
// barrier.  Matrices are row-major pairs in shared memory.

// (X^T Z)(i, j) = sum_p X[p][i] Z[p][j] over the rows p of X and Z (both
// rows x cols); tri: X is lower triangular, so p starts at i.  Two
// interleaved sums (the two_sum chain of one sum is serial).
__device__ __forceinline__ dd dd_tdot(const dd* X, const dd* Z, int rows, int cols, int i, int j, bool tri) {
  DDAcc a0, a1;
  a0.init0();
  a1.init0();
  int p = tri ? i : 0;
  const dd* x = X + (long long)p * cols + i;
  const dd* z = Z + (long long)p * cols + j;
  for (; p + 1 < rows; p += 2, x += 2 * cols, z += 2 * cols) {
    a0.fma(x[0], z[0]);
    a1.fma(x[cols], z[cols]);
  }
  if (p < rows) a0.fma(x[0], z[0]);
  return dd_add(a0.value(), a1.value());
}

// (W X)(i, j) = sum_{p <= i} W[i][p] X[p][j] for W lower triangular (ld w)
// and X with cols columns, two interleaved sums.
__device__ __forceinline__ dd dd_lmul(const dd* W, int w, const dd* X, int cols, int i, int j) {
  DDAcc a0, a1;
  a0.init0();
  a1.init0();
  const dd* wr = W + (long long)i * w;
  const dd* x = X + j;
  int p = 0;
  for (; p + 1 <= i; p += 2, x += 2 * cols) {
    a0.fma(wr[p], x[0]);
    a1.fma(wr[p + 1], x[cols]);
  }
  if (p <= i) a0.fma(wr[p], x[0]);
  return dd_add(a0.value(), a1.value());
}

// Element t of the lower triangle in row order: (i, j) with j <= i.
__device__ __forceinline__ void tri_ij(int t, int& i, int& j) {
  int r = __float2int_rz((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  if ((r + 1) * (r + 2) / 2 <= t) ++r;  // guard the float estimate
  if (r * (r + 1) / 2 > t) --r;
  i = r;
  j = t - r * (r + 1) / 2;
}

__device__ void load_dd(dd* dst, const double* src, int cnt) {
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) dst[t] = dd_from(src[t]);
}

__device__ void copy_dd(dd* dst, const dd* src, int cnt) {
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) dst[t] = src[t];
}

// dst (cols x rows) = src^T for src (rows x cols), row-major
__device__ void load_dd_t(dd* dst, const double* src, int rows, int cols) {
  for (int t = threadIdx.x; t < rows * cols; t += blockDim.x) {
    const int i = t / cols, j = t - i * cols;
    dst[j * rows + i] = dd_from(src[t]);
  }
}

__global__ void __launch_bounds__(kLqrThreads) k_lqr_schur(const __grid_constant__ LqrParams P) {
  extern __shared__ __align__(16) double lsm[];
  const LqrSeg sg = P.segs[blockIdx.x];
  const LqrDesc d = P.desc[sg.inst];
  const int n = d.n, m = d.m, N = d.N, nn = n * n, mm = m * m, mn = m * n;
  const int tid = threadIdx.x;
  dd* Wq = reinterpret_cast<dd*>(lsm);  // W = L^-1 of Q_k
  dd* At = Wq + nn;                     // A_k^T
  dd* Y = At + nn;                      // W A_k^T
  dd* C = Y + nn;                       // carry C_{k-1} (lower), then D_k in place
  dd* Wr = C + nn;                      // W_R of R_k
  dd* Bt = Wr + mm;                     // B_k^T (m x n)
  dd* V = Bt + mn;                      // W_R B_k^T
  dd* vq = V + mn;                      // q_k, then w_k
  dd* vt = vq + kLqrMax;                // t = W q_k
  dd* vr = vt + kLqrMax;                // r_k
  dd* vs = vr + kLqrMax;                // s = W_R r_k
  dd* vg = vs + kLqrMax;                // g_{k-1}
  const bool fused = P.hinst != nullptr;
  const InstDesc hd = fused ? P.hinst[sg.inst] : InstDesc{};
  const float inv_n = 1.0f / (float)n;
  const int ntri = n * (n + 1) / 2;
  for (int k = sg.a > 0 ? sg.a - 1 : 0; k < sg.b; ++k) {
    const bool own = k >= sg.a;  // row a-1 of a later segment only rebuilds the carry
    const bool hasA = k < N - 1;
    copy_dd(Wq, P.WQ + d.oQ + (long long)k * nn, nn);
    load_dd(vq, P.q + d.ov + (long long)k * n, n);
    if (hasA) {
      load_dd_t(At, P.A + d.oA + (long long)k * nn, n, n);
      load_dd_t(Bt, P.Bm + d.oB + (long long)k * n * m, n, m);
      copy_dd(Wr, P.WR + d.oR + (long long)k * mm, mm);
      load_dd(vr, P.r + d.ou + (long long)k * m, m);
    }
    __syncthreads();
    // t = W q_k, s = W_R r_k; then w_k = W^T t (into vq)
    for (int i = tid; i < n + (hasA ? m : 0); i += blockDim.x) {
      DDAcc a;
      a.init0();
      if (i < n) {
        for (int p = 0; p <= i; ++p) a.fma(Wq[i * n + p], vq[p]);
        vt[i] = a.value();
      } else {
        const int ir = i - n;
        for (int p = 0; p <= ir; ++p) a.fma(Wr[ir * m + p], vr[p]);
        vs[ir] = a.value();
      }
    }
    __syncthreads();
    for (int i = tid; i < n; i += blockDim.x) {
      DDAcc a;
      a.init0();
      for (int p = i; p < n; ++p) a.fma(Wq[p * n + i], vt[p]);
      vq[i] = a.value();
    }
    if (hasA) {  // Y = W A_k^T, V = W_R B_k^T (one pass over both)
      for (int t = tid; t < nn + mn; t += blockDim.x) {
        if (t < nn) {
          const int i = qdiv(t, inv_n), j = t - i * n;
          Y[t] = dd_lmul(Wq, n, At, n, i, j);
        } else {
          const int u = t - nn, i = qdiv(u, inv_n), j = u - i * n;
          V[u] = dd_lmul(Wr, m, Bt, n, i, j);
        }
      }
    }
    __syncthreads();
    if (own) {
      // O_k = -W^T Y, one row of O per run of threads (the same triangular
      // length across a warp); for a handle it goes through At (free once Y
      // is formed) so that the column-major slots are written coalesced
      if (hasA) {
        double* Oc = P.O ? P.O + d.oA + (long long)k * nn : nullptr;
        for (int t = tid; t < nn; t += blockDim.x) {
          const int a = qdiv(t, inv_n), c = t - a * n;  // element (a, c)
          const dd o = dd_neg(dd_tdot(Wq, Y, n, n, a, c, true));
          if (Oc) Oc[t] = dd_to(o);
          if (fused) At[t] = o;
        }
        if (fused) {
          __syncthreads();
          double* O64 = P.hO64 + hd.off64 + (long long)k * hd.bs64;
          float* O32 = P.hO32 + hd.off32 + (long long)k * hd.bs32;
          for (int t = tid; t < nn; t += blockDim.x) {  // t = c n + a
            const int c = qdiv(t, inv_n), a = t - c * n;
            const double ov = dd_to(At[a * n + c]);
            O64[t] = ov;
            O32[t] = d2f_rn(ov);  // the float32 copy rounds the float64 value, as bt_refactor's does
          }
        }
      }
      // D_k = W^T W + C_{k-1} (lower, in place), gamma_k
      for (int t = tid; t < ntri; t += blockDim.x) {
        int i, j;
        tri_ij(t, i, j);
        dd v = dd_tdot(Wq, Wq, n, n, i, j, true);
        if (k > 0) v = dd_add(v, C[i * n + j]);
        C[i * n + j] = v;
      }
      for (int i = tid; i < n; i += blockDim.x) {
        dd v = dd_add(dd_from(P.c[d.ov + (long long)k * n + i]), vq[i]);
        if (k > 0) v = dd_add(v, dd_neg(vg[i]));
        P.gamma[d.ov + (long long)k * n + i] = -dd_to(v);
      }
      __syncthreads();
      double* Dc = P.D ? P.D + d.oQ + (long long)k * nn : nullptr;
      double* D64 = fused ? P.hD64 + hd.off64 + (long long)k * hd.bs64 : nullptr;
      float* D32 = fused ? P.hD32 + hd.off32 + (long long)k * hd.bs32 : nullptr;
      for (int t = tid; t < nn; t += blockDim.x) {  // symmetric: both layouts index alike
        const int i = qdiv(t, inv_n), j = t - i * n;
        const dd v = C[j > i ? j * n + i : t];
        const double dv = dd_to(v);
        if (Dc) Dc[t] = dv;
        if (fused) {
          D64[t] = dv;
          D32[t] = d2f_rn(dv);
        }
      }
      __syncthreads();
    }
    if (hasA) {
      // C_k = Y^T Y + V^T V (lower), g_k = Y^T t + V^T s
      for (int t = tid; t < ntri; t += blockDim.x) {
        int i, j;
        tri_ij(t, i, j);
        C[i * n + j] = dd_add(dd_tdot(Y, Y, n, n, i, j, false), dd_tdot(V, V, m, n, i, j, false));
      }
      for (int i = tid; i < n; i += blockDim.x) {
        DDAcc a;
        a.init0();
        for (int p = 0; p < n; ++p) a.fma(Y[p * n + i], vt[p]);
        for (int p = 0; p < m; ++p) a.fma(V[p * n + i], vs[p]);
        vg[i] = a.value();
      }
    }
    __syncthreads();
  }
}

// ---- recovery ----------------------------------------------------------------
// Solve M y = v in place (v in `v`) with the Cholesky factor in lower(M).
__device__ void chol_solve(const double* M, double* v, int n, const double* rinv) {
  for (int j = 0; j < n; ++j) {  // L y = v
    if (threadIdx.x == 0) v[j] *= rinv[j];
    __syncthreads();
    const double yj = v[j];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) v[i] = fma(-M[i * n + j], yj, v[i]);
    __syncthreads();
  }
  for (int j = n - 1; j >= 0; --j) {  // L^T x = y
    if (threadIdx.x == 0) v[j] *= rinv[j];
    __syncthreads();
    const double xj = v[j];
    for (int i = threadIdx.x; i < j; i += blockDim.x) v[i] = fma(-M[j * n + i], xj, v[i]);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kLqrThreads) k_lqr_recover(const __grid_constant__ LqrParams P) {
  extern __shared__ __align__(16) double lsm[];
  const LqrSeg sg = P.segs[blockIdx.x];
  const LqrDesc d = P.desc[sg.inst];
  const int n = d.n, m = d.m, N = d.N, nn = n * n;
  double* L = lsm;                         // Q_k (n x n), then R_k (m x m)
  double* v = L + max(nn, m * m);
  double* rinv = v + kLqrMax;
  for (int k = sg.a; k < sg.b; ++k) {
    // x_k = -Q_k^-1 (q_k + lam_k - A_k^T lam_{k+1})
    load(L, P.Q + d.oQ + (long long)k * nn, nn);
    const double* lk = P.lam + d.ov + (long long)k * n;
    const double* lk1 = lk + n;
    const double* Ak = P.A + d.oA + (long long)k * nn;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double s = P.q[d.ov + (long long)k * n + i] + lk[i];
      if (k < N - 1)
        for (int p = 0; p < n; ++p) s = fma(-Ak[p * n + i], lk1[p], s);
      v[i] = s;
    }
    if (!chol(L, n, rinv)) { refuse(P, sg.inst, k, 0); return; }
    chol_solve(L, v, n, rinv);
    for (int i = threadIdx.x; i < n; i += blockDim.x) P.x[d.ov + (long long)k * n + i] = -v[i];
    __syncthreads();
    if (k < N - 1) {
      // u_k = -R_k^-1 (r_k - B_k^T lam_{k+1})
      load(L, P.R + d.oR + (long long)k * m * m, m * m);
      const double* Bk = P.Bm + d.oB + (long long)k * n * m;
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double s = P.r[d.ou + (long long)k * m + i];
        for (int p = 0; p < n; ++p) s = fma(-Bk[p * m + i], lk1[p], s);
        v[i] = s;
      }
      if (!chol(L, m, rinv)) { refuse(P, sg.inst, k, 1); return; }
      chol_solve(L, v, m, rinv);
      for (int i = threadIdx.x; i < m; i += blockDim.x) P.u[d.ou + (long long)k * m + i] = -v[i];
      __syncthreads();
    }
  }
}


// Recovery from the factors the formation left (W = L^-1 of Q_k and R_k, in
// pairs): one warp per knot k,
//   v = q_k + lam_k - A_k^T lam_{k+1},   x_k = -W^T (W v),
//   w = r_k - B_k^T lam_{k+1},           u_k = -W_R^T (W_R w),
// v and w in float64, the two triangular products in pairs with W staged in
// shared memory (row-major, lower); lane = row of W v and column of W^T t.
// No factorization, so no pivot to refuse.
constexpr int kRecWarps = 4;

__device__ void warp_wtw(const dd* Wg, dd* W, dd* v, dd* t, int n, int lane, double* out) {
  for (int e = lane; e < n * n; e += 32) W[e] = Wg[e];
  __syncwarp();
  for (int i = lane; i < n; i += 32) {  // t = W v
    DDAcc a;
    a.init0();
    for (int p = 0; p <= i; ++p) a.fma(W[i * n + p], v[p]);
    t[i] = a.value();
  }
  __syncwarp();
  for (int i = lane; i < n; i += 32) {  // out = -W^T t
    DDAcc a;
    a.init0();
    for (int p = i; p < n; ++p) a.fma(W[p * n + i], t[p]);
    out[i] = -dd_to(a.value());
  }
  __syncwarp();
}

__global__ void __launch_bounds__(kRecWarps * 32) k_lqr_recover_w(const __grid_constant__ LqrParams P, long long nknot,
                                                                   int B, int maxd) {
  extern __shared__ __align__(16) double lsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long task = (long long)blockIdx.x * kRecWarps + warp;
  if (task >= nknot) return;
  int lo = 0, hi = B - 1;  // the problem: last k with desc[k].okn <= task
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P.desc[mid].okn <= task) lo = mid;
    else hi = mid - 1;
  }
  const LqrDesc d = P.desc[lo];
  const int k = (int)(task - d.okn), n = d.n, m = d.m, N = d.N;
  dd* W = reinterpret_cast<dd*>(lsm) + (size_t)warp * (maxd * maxd + 2 * maxd);
  dd* v = W + maxd * maxd;
  dd* t = v + maxd;
  const double* lk = P.lam + d.ov + (long long)k * n;
  const double* lk1 = lk + n;
  // the right-hand sides in float64 (n^2 multiply-adds per knot, coalesced
  // down the columns of A_k), split into pairs once
  for (int i = lane; i < n; i += 32) {  // v = q_k + lam_k - A_k^T lam_{k+1}
    double a = P.q[d.ov + (long long)k * n + i] + lk[i];
    if (k < N - 1) {
      const double* Ak = P.A + d.oA + (long long)k * n * n;
      for (int p = 0; p < n; ++p) a = fma(-Ak[p * n + i], lk1[p], a);
    }
    v[i] = dd_from(a);
  }
  __syncwarp();
  warp_wtw(P.WQ + d.oQ + (long long)k * n * n, W, v, t, n, lane, P.x + d.ov + (long long)k * n);
  if (k < N - 1) {
    for (int i = lane; i < m; i += 32) {  // w = r_k - B_k^T lam_{k+1}
      double a = P.r[d.ou + (long long)k * m + i];
      const double* Bk = P.Bm + d.oB + (long long)k * n * m;
      for (int p = 0; p < n; ++p) a = fma(-Bk[p * m + i], lk1[p], a);
      v[i] = dd_from(a);
    }
    __syncwarp();
    warp_wtw(P.WR + d.oR + (long long)k * m * m, W, v, t, m, lane, P.u + d.ou + (long long)k * m);
  }
}

}  // namespace bt

namespace {

int smem_schur(int n, int m) { return (4 * n * n + m * m + 2 * n * m + 5 * bt::kLqrMax) * 8; }
int smem_recover(int n, int m) { return (std::max(n * n, m * m) + 2 * bt::kLqrMax) * 8; }

// Host descriptors and segments; checks the shapes.  Also the task count of
// k_lqr_winv and the element counts of Q and R (the sizes of its scratch).
bt_status lqr_plan(int B, const int* N, const int* n, const int* m, std::vector<bt::LqrDesc>& desc,
                   std::vector<bt::LqrSeg>& segs, int& maxn, int& maxm, long long& ntask, long long& nQ,
                   long long& nR) {
  if (B < 1 || !N || !n || !m) return BT_ERR_ARG;
  desc.resize(B);
  long long oA = 0, oB = 0, oQ = 0, oR = 0, ov = 0, ou = 0, ot = 0, okn = 0;
  maxn = maxm = 1;
  for (int k = 0; k < B; ++k) {
    if (N[k] < 1 || n[k] < 1 || n[k] > bt::kLqrMax || m[k] < 1 || m[k] > bt::kLqrMax) return BT_ERR_ARG;
    const long long Nk = N[k], nk = n[k], mk = m[k];
    desc[k] = bt::LqrDesc{N[k], n[k], m[k], 0, oA, oB, oQ, oR, ov, ou, ot, okn};
    oA += (Nk - 1) * nk * nk;
    oB += (Nk - 1) * nk * mk;
    oQ += Nk * nk * nk;
    oR += (Nk - 1) * mk * mk;
    ov += Nk * nk;
    ou += (Nk - 1) * mk;
    ot += 2 * Nk - 1;
    okn += Nk;
    maxn = std::max(maxn, n[k]);
    maxm = std::max(maxm, m[k]);
    for (int a = 0; a < N[k]; a += bt::kLqrSeg) segs.push_back(bt::LqrSeg{k, a, std::min(N[k], a + bt::kLqrSeg), 0});
  }
  ntask = ot;
  nQ = oQ;
  nR = oR;
  return BT_OK;
}

// Bytes of the device buffer a formation call uses: descriptors, segments
// and the failure key, then the W scratch of k_lqr_winv.
size_t lqr_head_bytes(size_t ndesc, size_t nsegs) {
  return ((ndesc * sizeof(bt::LqrDesc) + nsegs * sizeof(bt::LqrSeg) + 8 + 255) / 256) * 256;
}

// pre, pre_bytes: a caller-owned device buffer to use instead of a
// stream-ordered allocation (the handle-attached formation keeps one); with
// pre_bytes too small (or pre null) the call allocates, and *need (if
// non-null) receives the bytes it wanted.
bt_status lqr_run(bool schur, int B, const int* N, const int* n, const int* m, bt::LqrParams P, void* stream,
                  int* bad_inst, int* bad_row, char* pre = nullptr, size_t pre_bytes = 0, size_t* need = nullptr) {
  std::vector<bt::LqrDesc> desc;
  std::vector<bt::LqrSeg> segs;
  int maxn = 0, maxm = 0;
  long long ntask = 0, nQ = 0, nR = 0;
  bt_status s = lqr_plan(B, N, n, m, desc, segs, maxn, maxm, ntask, nQ, nR);
  if (s != BT_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bd = desc.size() * sizeof(bt::LqrDesc), bs = segs.size() * sizeof(bt::LqrSeg);
  const size_t head = lqr_head_bytes(desc.size(), segs.size());
  const size_t scratch = schur ? (size_t)(nQ + nR) * sizeof(bt::dd) : 0;
  if (need) *need = head + scratch;
  const bool own_buf = !(pre && pre_bytes >= head + scratch);
  char* buf = own_buf ? nullptr : pre;
  if (own_buf && cudaMallocAsync((void**)&buf, head + scratch, st) != cudaSuccess) return BT_ERR_ALLOC;
  const auto ok = [](cudaError_t e) { return e == cudaSuccess; };
  bt_status out = BT_OK;
  unsigned long long key = ~0ull;
  P.desc = reinterpret_cast<const bt::LqrDesc*>(buf);
  P.segs = reinterpret_cast<const bt::LqrSeg*>(buf + bd);
  P.fail_key = reinterpret_cast<unsigned long long*>(buf + ((bd + bs + 7) / 8) * 8);
  P.WQ = reinterpret_cast<bt::dd*>(buf + head);
  P.WR = P.WQ + nQ;
  const int smem = schur ? smem_schur(maxn, maxm) : smem_recover(maxn, maxm);
  const void* fn = schur ? (const void*)bt::k_lqr_schur : (const void*)bt::k_lqr_recover;
  const int maxd = std::max(maxn, maxm);
  const int wstride = maxd * maxd + maxd;  // pairs per warp of k_lqr_winv: one block and its pivots
  const int wsmem = bt::kWinvWarps * wstride * (int)sizeof(bt::dd);
  if (!ok(cudaMemcpyAsync(buf, desc.data(), bd, cudaMemcpyHostToDevice, st)) ||
      !ok(cudaMemcpyAsync(buf + bd, segs.data(), bs, cudaMemcpyHostToDevice, st)) ||
      !ok(cudaMemsetAsync(P.fail_key, 0xff, sizeof(unsigned long long), st)) ||
      !ok(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) ||
      (schur && !ok(cudaFuncSetAttribute(bt::k_lqr_winv, cudaFuncAttributeMaxDynamicSharedMemorySize, wsmem)))) {
    out = BT_ERR_CUDA;
  } else {
    if (schur) {
      const long long wgrid = (ntask + bt::kWinvWarps - 1) / bt::kWinvWarps;
      bt::k_lqr_winv<<<(unsigned)wgrid, bt::kWinvWarps * 32, wsmem, st>>>(P, ntask, B, wstride);
      if (!ok(cudaGetLastError())) out = BT_ERR_CUDA;
    }
    void* args[] = {(void*)&P};
    if (out != BT_OK ||
        !ok(cudaLaunchKernel(fn, dim3((unsigned)segs.size()), dim3(bt::kLqrThreads), args, smem, st)) ||
        !ok(cudaMemcpyAsync(&key, P.fail_key, sizeof(key), cudaMemcpyDeviceToHost, st)) ||
        !ok(cudaStreamSynchronize(st)))
      out = BT_ERR_CUDA;
  }
  if (own_buf) cudaFreeAsync(buf, st);
  if (out == BT_OK && key != ~0ull) {
    if (bad_inst) *bad_inst = (int)(key >> 32);
    if (bad_row) *bad_row = (int)((key & 0xffffffffu) >> 1);
    out = BT_ERR_NOT_SPD;
  }
  return out;
}

bool any_long(int B, const int* N) {
  if (B < 1 || !N) return false;
  for (int k = 0; k < B; ++k)
    if (N[k] > 1) return true;
  return false;
}

}  // namespace

extern "C" bt_status bt_lqr_schur(int B, const int* N, const int* n, const int* m, const double* A,
                                  const double* Bm, const double* Q, const double* R, const double* q,
                                  const double* r, const double* c, double* D, double* O, double* gamma,
                                  void* stream, int* bad_inst, int* bad_row) {
  if (!Q || !q || !c || !D || !gamma) return BT_ERR_ARG;
  if (any_long(B, N) && (!A || !Bm || !R || !r || !O)) return BT_ERR_ARG;
  bt::LqrParams P{};
  P.A = A; P.Bm = Bm; P.Q = Q; P.R = R; P.q = q; P.r = r; P.c = c;
  P.D = D; P.O = O; P.gamma = gamma;
  return lqr_run(true, B, N, n, m, P, stream, bad_inst, bad_row);
}

// The formation into a mixed handle's block arrays (D, O in float64 and
// float32; column-major slots at the handle's offsets), for
// bt_lqr_refactor, in the caller's device buffer (buf, buf_bytes) when it is
// large enough; *need receives the bytes a call uses.  Shapes are the
// handle's; the caller checks them.
extern "C" bt_status bt_lqr_schur_handle(int B, const int* N, const int* n, const int* m, const double* A,
                                         const double* Bm, const double* Q, const double* R, const double* q,
                                         const double* r, const double* c, double* gamma, const bt::InstDesc* hinst,
                                         double* hD64, double* hO64, float* hD32, float* hO32, float* hDinv32,
                                         void* stream, int* bad_inst, int* bad_row, void* buf, size_t buf_bytes,
                                         size_t* need) {
  if (!Q || !q || !c || !gamma || !hinst || !hD64 || !hD32 || !hDinv32) return BT_ERR_ARG;
  if (any_long(B, N) && (!A || !Bm || !R || !r || !hO64 || !hO32)) return BT_ERR_ARG;
  bt::LqrParams P{};
  P.A = A; P.Bm = Bm; P.Q = Q; P.R = R; P.q = q; P.r = r; P.c = c;
  P.gamma = gamma;
  P.hinst = hinst;
  P.hD64 = hD64; P.hO64 = hO64; P.hD32 = hD32; P.hO32 = hO32; P.hDinv32 = hDinv32;
  return lqr_run(true, B, N, n, m, P, stream, bad_inst, bad_row, static_cast<char*>(buf), buf_bytes, need);
}

// Bytes of the device buffer bt_lqr_schur_handle uses for these shapes (0 on
// bad shapes): the handle allocates it once and keeps it, and the factors W
// it holds serve bt_lqr_recover_factored.
extern "C" size_t bt_lqr_handle_bytes(int B, const int* N, const int* n, const int* m) {
  std::vector<bt::LqrDesc> desc;
  std::vector<bt::LqrSeg> segs;
  int maxn = 0, maxm = 0;
  long long ntask = 0, nQ = 0, nR = 0;
  if (lqr_plan(B, N, n, m, desc, segs, maxn, maxm, ntask, nQ, nR) != BT_OK) return 0;
  return lqr_head_bytes(desc.size(), segs.size()) + (size_t)(nQ + nR) * sizeof(bt::dd);
}

// The recovery from the W factors in buf (left there by bt_lqr_schur_handle
// for the same shapes).  Synchronises.
extern "C" bt_status bt_lqr_recover_w_run(int B, const int* N, const int* n, const int* m, const double* A,
                                          const double* Bm, const double* q, const double* r, const double* lambda,
                                          double* x, double* u, const void* buf, void* stream) {
  if (!q || !lambda || !x || !buf) return BT_ERR_ARG;
  if (any_long(B, N) && (!A || !Bm || !r || !u)) return BT_ERR_ARG;
  std::vector<bt::LqrDesc> desc;
  std::vector<bt::LqrSeg> segs;
  int maxn = 0, maxm = 0;
  long long ntask = 0, nQ = 0, nR = 0;
  bt_status s = lqr_plan(B, N, n, m, desc, segs, maxn, maxm, ntask, nQ, nR);
  if (s != BT_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long nknot = desc.back().okn + desc.back().N;
  bt::LqrParams P{};
  P.A = A; P.Bm = Bm; P.q = q; P.r = r; P.lam = lambda; P.x = x; P.u = u;
  P.WQ = reinterpret_cast<bt::dd*>(const_cast<char*>(static_cast<const char*>(buf)) +
                                   lqr_head_bytes(desc.size(), segs.size()));
  P.WR = P.WQ + nQ;
  const size_t bd = desc.size() * sizeof(bt::LqrDesc);
  char* dbuf = nullptr;
  if (cudaMallocAsync((void**)&dbuf, bd, st) != cudaSuccess) return BT_ERR_ALLOC;
  P.desc = reinterpret_cast<const bt::LqrDesc*>(dbuf);
  const int maxd = std::max(maxn, maxm);
  const int smem = bt::kRecWarps * (maxd * maxd + 2 * maxd) * (int)sizeof(bt::dd);
  const auto ok = [](cudaError_t e) { return e == cudaSuccess; };
  bt_status out = BT_OK;
  if (!ok(cudaMemcpyAsync(dbuf, desc.data(), bd, cudaMemcpyHostToDevice, st)) ||
      !ok(cudaFuncSetAttribute(bt::k_lqr_recover_w, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
    out = BT_ERR_CUDA;
  else {
    bt::k_lqr_recover_w<<<(unsigned)((nknot + bt::kRecWarps - 1) / bt::kRecWarps), bt::kRecWarps * 32, smem, st>>>(
        P, nknot, B, maxd);
    if (!ok(cudaGetLastError())) out = BT_ERR_CUDA;
  }
  cudaFreeAsync(dbuf, st);
  if (!ok(cudaStreamSynchronize(st)) && out == BT_OK) out = BT_ERR_CUDA;
  return out;
}

extern "C" bt_status bt_lqr_recover(int B, const int* N, const int* n, const int* m, const double* A,
                                    const double* Bm, const double* Q, const double* R, const double* q,
                                    const double* r, const double* lambda, double* x, double* u, void* stream) {
  if (!Q || !q || !lambda || !x) return BT_ERR_ARG;
  if (any_long(B, N) && (!A || !Bm || !R || !r || !u)) return BT_ERR_ARG;
  bt::LqrParams P{};
  P.A = A; P.Bm = Bm; P.Q = Q; P.R = R; P.q = q; P.r = r; P.lam = lambda;
  P.x = x; P.u = u;
  return lqr_run(false, B, N, n, m, P, stream, nullptr, nullptr);
}
