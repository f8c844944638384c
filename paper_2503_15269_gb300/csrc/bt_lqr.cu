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
// Float64 throughout (the blocks feed the float64 residual of the solver).
// One CTA walks a segment of consecutive block rows of one instance and
// carries A_{k-1}, P_{k-1}, w_{k-1} in shared memory from row to row, so each
// row inverts one Q_k (Cholesky, W = L^-1, W^T W) and forms one n x n product
// P_k and one symmetric A_{k-1} P_{k-1}.  Float64 issues at ~2 FMA per clock
// per SM on GB300, so these kernels are bound by the float64 pipe.
#include <algorithm>
#include <vector>

#include "../../include/bt.h"
#include "bt_common.cuh"

namespace bt {

constexpr int kLqrThreads = 128;
constexpr int kLqrSeg = 16;  // block rows per CTA segment
constexpr int kLqrMax = 48;  // largest n and m (shared-memory budget)
static_assert(kLqrThreads >= kLqrMax, "one thread per row of a block column");

struct LqrDesc {
  int N, n, m, pad;
  long long oA, oB, oQ, oR, ov, ou;  // element offsets: A/O, Bm, Q/D, R, n-vectors, m-vectors
};
struct LqrSeg {
  int inst, a, b, pad;
};

struct LqrParams {
  const LqrDesc* desc;
  const LqrSeg* segs;
  const double *A, *Bm, *Q, *R, *q, *r, *c, *lam;
  double *D, *O, *gamma, *x, *u;
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

// From the Cholesky factor in lower(M): M <- M^-1 = W^T W with W = L^-1.
// W by right-looking forward substitution on the columns of I, two barriers
// per row: row j of B (I minus the earlier updates) is scaled to W_j by
// 1/L_jj, then the rows below take one FMA per element.
__device__ void chol_inverse(double* M, double* W, int n, const double* rinv) {
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) W[t] = (t / n == t % n) ? 1.0 : 0.0;
  for (int j = 0; j < n; ++j) {
    __syncthreads();
    if (threadIdx.x <= j) W[j * n + threadIdx.x] *= rinv[j];
    __syncthreads();
    const int cols = j + 1, rows = n - j - 1;
    for (int t = threadIdx.x; t < rows * cols; t += blockDim.x) {
      const int i = j + 1 + t / cols, c = t % cols;
      W[i * n + c] = fma(-M[i * n + j], W[j * n + c], W[i * n + c]);
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int i = t / n, j = t % n;
    if (j > i) continue;
    double acc = 0.0;
    for (int r = i; r < n; ++r) acc = fma(W[r * n + i], W[r * n + j], acc);
    M[i * n + j] = acc;
    M[j * n + i] = acc;
  }
  __syncthreads();
}

// C (+)= X Y^T for X [rows x k], Y [cols x k] (row-major, leading dims k);
// sym: C is symmetric, only j <= i is computed and mirrored.
__device__ void gemm_nt(double* C, int ldc, const double* X, const double* Y, int rows, int cols, int k, double s,
                        bool acc, bool sym) {
  for (int t = threadIdx.x; t < rows * cols; t += blockDim.x) {
    const int i = t / cols, j = t % cols;
    if (sym && j > i) continue;
    double v = 0.0;
    for (int p = 0; p < k; ++p) v = fma(X[i * k + p], Y[j * k + p], v);
    v *= s;
    const double o = acc ? C[i * ldc + j] + v : v;
    C[i * ldc + j] = o;
    if (sym && j < i) C[j * ldc + i] = o;
  }
  __syncthreads();
}

__device__ void load(double* dst, const double* src, int cnt) {
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) dst[t] = src[t];
}

__device__ void refuse(const LqrParams& P, int inst, int row, int isR) {
  if (threadIdx.x == 0)
    atomicMin(P.fail_key, ((unsigned long long)inst << 32) | (unsigned)(2 * row + isR));
}

// ---- formation ---------------------------------------------------------------
__global__ void __launch_bounds__(kLqrThreads) k_lqr_schur(const __grid_constant__ LqrParams P) {
  extern __shared__ __align__(16) double lsm[];
  const LqrSeg sg = P.segs[blockIdx.x];
  const LqrDesc d = P.desc[sg.inst];
  const int n = d.n, m = d.m, N = d.N, nn = n * n;
  double* Qi = lsm;             // Q_k^-1
  double* Ak = Qi + nn;         // A_k
  double* Pk = Ak + nn;         // P_k = Q_k^-1 A_k^T
  double* Ap = Pk + nn;         // A_{k-1}
  double* Pp = Ap + nn;         // P_{k-1}
  double* Wd = Pp + nn;         // inverse scratch, then the D accumulator
  double* Ri = Wd + nn;         // R_{k-1}^-1  (m x m)
  double* Rw = Ri + m * m;      // its scratch
  double* Bk = Rw + m * m;      // B_{k-1}     (n x m)
  double* Uk = Bk + n * m;      // B_{k-1} R_{k-1}^-1 (n x m)
  double* wk = Uk + n * m;      // w_k = Q_k^-1 q_k
  double* wp = wk + kLqrMax;    // w_{k-1}
  double* rinv = wp + kLqrMax;  // reciprocal pivots
  const double* Qb = P.Q + d.oQ;
  const double* Ab = P.A + d.oA;
  const double* qb = P.q + d.ov;
  // Q_k^-1, A_k, P_k, w_k of row k into (Qi, Ak, Pk, wk); false if Q_k is refused
  auto row_terms = [&](int k) -> bool {
    load(Qi, Qb + (long long)k * nn, nn);
    if (!chol(Qi, n, rinv)) return false;
    chol_inverse(Qi, Wd, n, rinv);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double v = 0.0;
      for (int p = 0; p < n; ++p) v = fma(Qi[i * n + p], qb[(long long)k * n + p], v);
      wk[i] = v;
    }
    if (k < N - 1) {
      load(Ak, Ab + (long long)k * nn, nn);
      __syncthreads();
      gemm_nt(Pk, n, Qi, Ak, n, n, n, 1.0, false, false);  // Q_k^-1 A_k^T (Q_k^-1 symmetric)
    }
    __syncthreads();
    return true;
  };
  auto carry = [&]() {  // (Ak, Pk, wk) of row k become (Ap, Pp, wp)
    for (int t = threadIdx.x; t < nn; t += blockDim.x) {
      Ap[t] = Ak[t];
      Pp[t] = Pk[t];
    }
    for (int t = threadIdx.x; t < n; t += blockDim.x) wp[t] = wk[t];
    __syncthreads();
  };
  if (sg.a > 0) {
    if (!row_terms(sg.a - 1)) { refuse(P, sg.inst, sg.a - 1, 0); return; }
    carry();
  }
  for (int k = sg.a; k < sg.b; ++k) {
    if (!row_terms(k)) { refuse(P, sg.inst, k, 0); return; }
    double* Dk = P.D + d.oQ + (long long)k * nn;
    double* gk = P.gamma + d.ov + (long long)k * n;
    const double* ck = P.c + d.ov + (long long)k * n;
    if (k < N - 1) {
      double* Ok = P.O + d.oA + (long long)k * nn;
      for (int t = threadIdx.x; t < nn; t += blockDim.x) Ok[t] = -Pk[t];
    }
    if (k == 0) {
      for (int t = threadIdx.x; t < nn; t += blockDim.x) Dk[t] = Qi[t];
      for (int t = threadIdx.x; t < n; t += blockDim.x) gk[t] = -(ck[t] + wk[t]);
    } else {
      // D_k = Q_k^-1 + A_{k-1} P_{k-1} + (B R^-1) B^T over row k-1's input
      for (int t = threadIdx.x; t < nn; t += blockDim.x) Wd[t] = Qi[t];
      __syncthreads();
      // A_{k-1} P_{k-1} = A_{k-1} Q^-1 A_{k-1}^T: symmetric; (A P)[i][j] = sum_p A[i][p] P[p][j]
      for (int t = threadIdx.x; t < nn; t += blockDim.x) {
        const int i = t / n, j = t % n;
        if (j > i) continue;
        double v = 0.0;
        for (int p = 0; p < n; ++p) v = fma(Ap[i * n + p], Pp[p * n + j], v);
        Wd[i * n + j] += v;
        if (j < i) Wd[j * n + i] += v;
      }
      __syncthreads();
      const double* Rb = P.R + d.oR + (long long)(k - 1) * m * m;
      load(Ri, Rb, m * m);
      load(Bk, P.Bm + d.oB + (long long)(k - 1) * n * m, n * m);
      if (!chol(Ri, m, rinv)) { refuse(P, sg.inst, k - 1, 1); return; }
      chol_inverse(Ri, Rw, m, rinv);
      // U = B R^-1 (R^-1 symmetric: U[i][j] = sum_p B[i][p] Ri[j][p])
      gemm_nt(Uk, m, Bk, Ri, n, m, m, 1.0, false, false);
      gemm_nt(Wd, n, Uk, Bk, n, n, m, 1.0, true, true);
      for (int t = threadIdx.x; t < nn; t += blockDim.x) Dk[t] = Wd[t];
      // gamma_k = -(c_k + w_k - A_{k-1} w_{k-1} - U r_{k-1})
      const double* rp = P.r + d.ou + (long long)(k - 1) * m;
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double v = ck[i] + wk[i];
        for (int p = 0; p < n; ++p) v = fma(-Ap[i * n + p], wp[p], v);
        for (int p = 0; p < m; ++p) v = fma(-Uk[i * m + p], rp[p], v);
        gk[i] = -v;
      }
    }
    __syncthreads();
    carry();
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

}  // namespace bt

namespace {

int smem_schur(int n, int m) { return (6 * n * n + 2 * m * m + 2 * n * m + 3 * bt::kLqrMax) * 8; }
int smem_recover(int n, int m) { return (std::max(n * n, m * m) + 2 * bt::kLqrMax) * 8; }

// Host descriptors and segments; checks the shapes.
bt_status lqr_plan(int B, const int* N, const int* n, const int* m, std::vector<bt::LqrDesc>& desc,
                   std::vector<bt::LqrSeg>& segs, int& maxn, int& maxm) {
  if (B < 1 || !N || !n || !m) return BT_ERR_ARG;
  desc.resize(B);
  long long oA = 0, oB = 0, oQ = 0, oR = 0, ov = 0, ou = 0;
  maxn = maxm = 1;
  for (int k = 0; k < B; ++k) {
    if (N[k] < 1 || n[k] < 1 || n[k] > bt::kLqrMax || m[k] < 1 || m[k] > bt::kLqrMax) return BT_ERR_ARG;
    const long long Nk = N[k], nk = n[k], mk = m[k];
    desc[k] = bt::LqrDesc{N[k], n[k], m[k], 0, oA, oB, oQ, oR, ov, ou};
    oA += (Nk - 1) * nk * nk;
    oB += (Nk - 1) * nk * mk;
    oQ += Nk * nk * nk;
    oR += (Nk - 1) * mk * mk;
    ov += Nk * nk;
    ou += (Nk - 1) * mk;
    maxn = std::max(maxn, n[k]);
    maxm = std::max(maxm, m[k]);
    for (int a = 0; a < N[k]; a += bt::kLqrSeg) segs.push_back(bt::LqrSeg{k, a, std::min(N[k], a + bt::kLqrSeg), 0});
  }
  return BT_OK;
}

bt_status lqr_run(bool schur, int B, const int* N, const int* n, const int* m, bt::LqrParams P, void* stream,
                  int* bad_inst, int* bad_row) {
  std::vector<bt::LqrDesc> desc;
  std::vector<bt::LqrSeg> segs;
  int maxn = 0, maxm = 0;
  bt_status s = lqr_plan(B, N, n, m, desc, segs, maxn, maxm);
  if (s != BT_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bd = desc.size() * sizeof(bt::LqrDesc), bs = segs.size() * sizeof(bt::LqrSeg);
  char* buf = nullptr;
  if (cudaMallocAsync((void**)&buf, bd + bs + 64, st) != cudaSuccess) return BT_ERR_ALLOC;
  const auto ok = [](cudaError_t e) { return e == cudaSuccess; };
  bt_status out = BT_OK;
  unsigned long long key = ~0ull;
  P.desc = reinterpret_cast<const bt::LqrDesc*>(buf);
  P.segs = reinterpret_cast<const bt::LqrSeg*>(buf + bd);
  P.fail_key = reinterpret_cast<unsigned long long*>(buf + ((bd + bs + 7) / 8) * 8);
  const int smem = schur ? smem_schur(maxn, maxm) : smem_recover(maxn, maxm);
  const void* fn = schur ? (const void*)bt::k_lqr_schur : (const void*)bt::k_lqr_recover;
  if (!ok(cudaMemcpyAsync(buf, desc.data(), bd, cudaMemcpyHostToDevice, st)) ||
      !ok(cudaMemcpyAsync(buf + bd, segs.data(), bs, cudaMemcpyHostToDevice, st)) ||
      !ok(cudaMemsetAsync(P.fail_key, 0xff, sizeof(unsigned long long), st)) ||
      !ok(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) {
    out = BT_ERR_CUDA;
  } else {
    void* args[] = {(void*)&P};
    if (!ok(cudaLaunchKernel(fn, dim3((unsigned)segs.size()), dim3(bt::kLqrThreads), args, smem, st)) ||
        !ok(cudaMemcpyAsync(&key, P.fail_key, sizeof(key), cudaMemcpyDeviceToHost, st)) ||
        !ok(cudaStreamSynchronize(st)))
      out = BT_ERR_CUDA;
  }
  cudaFreeAsync(buf, st);
  if (out == BT_OK && key != ~0ull) {
    if (bad_inst) *bad_inst = (int)(key >> 32);
    if (bad_row) *bad_row = (int)((key & 0xffffffffu) >> 1);
    out = BT_ERR_NOT_SPD;
  }
  return out;
}

}  // namespace

extern "C" bt_status bt_lqr_schur(int B, const int* N, const int* n, const int* m, const double* A,
                                  const double* Bm, const double* Q, const double* R, const double* q,
                                  const double* r, const double* c, double* D, double* O, double* gamma,
                                  void* stream, int* bad_inst, int* bad_row) {
  if (!Q || !q || !c || !D || !gamma) return BT_ERR_ARG;
  bt::LqrParams P{};
  P.A = A; P.Bm = Bm; P.Q = Q; P.R = R; P.q = q; P.r = r; P.c = c;
  P.D = D; P.O = O; P.gamma = gamma;
  return lqr_run(true, B, N, n, m, P, stream, bad_inst, bad_row);
}

extern "C" bt_status bt_lqr_recover(int B, const int* N, const int* n, const int* m, const double* A,
                                    const double* Bm, const double* Q, const double* R, const double* q,
                                    const double* r, const double* lambda, double* x, double* u, void* stream) {
  if (!Q || !q || !lambda || !x) return BT_ERR_ARG;
  bt::LqrParams P{};
  P.A = A; P.Bm = Bm; P.Q = Q; P.R = R; P.q = q; P.r = r; P.lam = lambda;
  P.x = x; P.u = u;
  return lqr_run(false, B, N, n, m, P, stream, nullptr, nullptr);
}
