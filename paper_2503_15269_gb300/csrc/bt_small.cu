// Small single instances (float64): the whole PCG of one instance in one CTA
// with every block resident in shared memory.
//
// For an instance as small as N = 16 block rows of n = 6 (the seven float64
// block arrays D, O, D^-1, E, Hd, Hu, Hl take 32 KB) the persistent kernel's
// bulk-copy pipeline costs more than the arithmetic: each sweep is one chunk,
// each chunk waits for its copy.  Here the blocks are loaded once per solve
// and every iteration runs from shared memory: block-tridiagonal SpMV
// (Eq. 1), the preconditioner apply y0 = G r, y_j = H y_{j-1},
// z = sum_j alpha_j y_j (Sec. 4.1-4.2 closed form), textbook PCG on the
// float64 user vectors with a fixed-order block reduction for the dots.
// Results and statuses are those of the persistent kernel's float64 path
// (recursive residual test ||r|| <= tol ||b||, x0 = 0 or the caller's).
#include <cstdint>

#include "../../include/bt.h"
#include "bt_common.cuh"

namespace bt {

constexpr int kSmallThreads = 256;
constexpr int kSmallMaxBytes = 200 * 1024;  // shared memory the engine may take

struct SmallParams {
  const double *D, *O, *Dinv, *E, *Hd, *Hu, *Hl;  // library slots (column-major, stride bs)
  int N, n, bs, m;
  double alpha[kMaxM];
  const double* b;
  double* x;
  int use_x0;
  double tol;
  int maxit;
  long long budget;
  double* hist;  // [maxit][3]: rel. residual, alpha_k, beta_k (or null)
  int hist_len;
  int *iters, *status, *outer;
  double *resid, *errval;
};

// Shared-memory floats of the engine: seven block arrays of N slots and eight
// vectors of N n doubles, plus the reduction scratch.
__host__ __device__ inline long long small_bytes(int N, int n, int bs) {
  return (7ll * N * bs + 8ll * N * n) * 8 + 64 * 8;
}

struct Small {
  const SmallParams& P;
  double *D, *O, *Dinv, *E, *Hd, *Hu, *Hl;
  double* red;  // [32] warp partials + broadcast
  int N, n, bs, tid, nel;

  __device__ Small(const SmallParams& P_, double* sm) : P(P_) {
    N = P.N;
    n = P.n;
    bs = P.bs;
    tid = threadIdx.x;
    nel = N * n;
    const long long A = (long long)N * bs;
    D = sm; O = D + A; Dinv = O + A; E = Dinv + A; Hd = E + A; Hu = Hd + A; Hl = Hu + A;
    red = Hl + A + 8ll * nel;
  }
  __device__ double* vec(int k) { return Hl + (long long)N * bs + (long long)k * nel; }

  // sum over the CTA, fixed order: a shuffle tree within each warp, then one
  // over the warps' sums (float64 adds are slow here; no serial chains)
  __device__ double reduce(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();  // red free (the previous broadcast was read)
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid < 32) {
      double w = tid < kSmallThreads / 32 ? red[tid] : 0.0;
#pragma unroll
      for (int o = kSmallThreads / 64; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
      if (tid == 0) red[32] = w;
    }
    __syncthreads();
    return red[32];
  }

  // out = (block row of M) v for every element (i, a); kind 0: S, 1: G, 2: H
  __device__ void sweep(int kind, const double* v, double* out) {
    for (int e = tid; e < nel; e += kSmallThreads) {
      const int i = e / n, a = e - i * n;
      const double* vi = v + i * n;
      double acc = 0.0;
      const double* M0 = (kind == 0 ? D : (kind == 1 ? Dinv : Hd)) + (long long)i * bs;
      for (int c = 0; c < n; ++c) acc = fma(M0[c * n + a], vi[c], acc);
      if (kind == 0 || kind == 1) {
        const double* M = kind == 0 ? O : E;
        const double sg = kind == 0 ? 1.0 : -1.0;  // G's off-diagonal blocks are -E_i, -E_{i-1}^T
        double t = 0.0;
        if (i + 1 < N) {  // (i, i+1): O_i / E_i
          const double* Mi = M + (long long)i * bs;
          const double* vn = vi + n;
          for (int c = 0; c < n; ++c) t = fma(Mi[c * n + a], vn[c], t);
        }
        if (i >= 1) {  // (i, i-1): O_{i-1}^T / E_{i-1}^T
          const double* Mp = M + (long long)(i - 1) * bs;
          const double* vp = vi - n;
          for (int c = 0; c < n; ++c) t = fma(Mp[a * n + c], vp[c], t);
        }
        acc = fma(sg, t, acc);
      } else {
        if (i + 2 < N) {  // (i, i+2): Hu_i
          const double* Mi = Hu + (long long)i * bs;
          const double* vn = vi + 2 * n;
          for (int c = 0; c < n; ++c) acc = fma(Mi[c * n + a], vn[c], acc);
        }
        if (i >= 2) {  // (i, i-2): Hl_{i-2}
          const double* Mp = Hl + (long long)(i - 2) * bs;
          const double* vp = vi - 2 * n;
          for (int c = 0; c < n; ++c) acc = fma(Mp[c * n + a], vp[c], acc);
        }
      }
      out[e] = acc;
    }
  }

  // z = M^-1 r (y0 = G r, y_j = H y_{j-1}, z = y0 + sum_{j>0} alpha_j y_j); returns r . z
  __device__ double precond(const double* r, double* z, double* y0, double* ya, double* yb) {
    sweep(1, r, P.m == 1 ? z : y0);
    __syncthreads();
    if (P.m > 1) {
      const double* yin = y0;
      for (int j = 1; j < P.m; ++j) {
        double* yout = (j & 1) ? ya : yb;
        sweep(2, yin, yout);
        __syncthreads();
        yin = yout;
        const double aj = P.alpha[j];
        for (int e = tid; e < nel; e += kSmallThreads) z[e] = fma(aj, yout[e], j == 1 ? y0[e] : z[e]);
        __syncthreads();
      }
    }
    double t = 0.0;
    for (int e = tid; e < nel; e += kSmallThreads) t = fma(r[e], z[e], t);
    return reduce(t);
  }
};

__global__ void __launch_bounds__(kSmallThreads, 1) bt_small_kernel(const __grid_constant__ SmallParams P) {
  extern __shared__ __align__(16) double smd[];
  Small Sm(P, smd);
  const int tid = threadIdx.x;
  const long long deadline = clock64() + P.budget;
  // load the blocks (all N slots of the seven arrays) once
  {
    const long long A = (long long)P.N * P.bs;
    const double* src[7] = {P.D, P.O, P.Dinv, P.E, P.Hd, P.Hu, P.Hl};
    double* dst[7] = {Sm.D, Sm.O, Sm.Dinv, Sm.E, Sm.Hd, Sm.Hu, Sm.Hl};
    const int na = P.m > 1 ? 7 : 4;
    for (int k = 0; k < na; ++k)
      for (long long t = tid; t < A; t += kSmallThreads) dst[k][t] = __ldg(src[k] + t);
  }
  const int nel = Sm.nel;
  double* x = Sm.vec(0);
  double* r = Sm.vec(1);
  double* p = Sm.vec(2);
  double* q = Sm.vec(3);
  double* z = Sm.vec(4);
  double* y0 = Sm.vec(5);
  double* ya = Sm.vec(6);
  double* yb = Sm.vec(7);
  double* const hist = (P.hist && tid == 0) ? P.hist : nullptr;
  auto record = [&](int idx, int field, double v) {
    if (hist && idx >= 0 && idx < P.hist_len) hist[(size_t)idx * 3 + field] = v;
  };
  // r0 = b - S x0 (or b with x0 = 0)
  double bb = 0.0;
  for (int e = tid; e < nel; e += kSmallThreads) {
    const double bv = P.b[e];
    bb = fma(bv, bv, bb);
    x[e] = P.use_x0 ? P.x[e] : 0.0;
    r[e] = bv;
  }
  __syncthreads();
  if (P.use_x0) {
    Sm.sweep(0, x, q);
    __syncthreads();
    for (int e = tid; e < nel; e += kSmallThreads) r[e] -= q[e];
  }
  const double nb = sqrt(Sm.reduce(bb));
  double rr_loc = 0.0;
  for (int e = tid; e < nel; e += kSmallThreads) rr_loc = fma(r[e], r[e], rr_loc);
  double rr = Sm.reduce(rr_loc);
  int status = kOK, it = 0;
  double errv = 0.0;
  const double nrhs = P.use_x0 ? nb : sqrt(rr);
  const double thr2 = (P.tol * nrhs) * (P.tol * nrhs);
  if (!isfinite(rr) || !isfinite(nb)) {
    status = kErrNonfinite;
  } else if (nrhs > 0.0 && !(rr <= thr2)) {
    double rho = Sm.precond(r, z, y0, ya, yb);
    for (int e = tid; e < nel; e += kSmallThreads) p[e] = z[e];
    __syncthreads();
    for (int k = 1;; ++k) {
      if (k > P.maxit) {
        status = kErrNoConv;
        it = P.maxit;
        break;
      }
      if (clock64() > deadline) {
        status = kErrTimeout;
        it = k - 1;
        break;
      }
      Sm.sweep(0, p, q);
      double t = 0.0;
      for (int e = tid; e < nel; e += kSmallThreads) t = fma(p[e], q[e], t);
      const double pq = Sm.reduce(t);
      if (!isfinite(pq)) {
        status = kErrNonfinite;
        it = k - 1;
        break;
      }
      if (!(pq > 0.0)) {
        status = kErrBreakdown;
        it = k - 1;
        errv = pq;
        break;
      }
      const double al = rho / pq;
      record(k - 1, 1, al);
      record(k - 1, 2, 0.0);
      t = 0.0;
      for (int e = tid; e < nel; e += kSmallThreads) {
        x[e] = fma(al, p[e], x[e]);
        const double rv = fma(-al, q[e], r[e]);
        r[e] = rv;
        t = fma(rv, rv, t);
      }
      rr = Sm.reduce(t);
      it = k;
      record(k - 1, 0, sqrt(rr) / nrhs);
      if (!isfinite(rr)) {
        status = kErrNonfinite;
        break;
      }
      if (rr <= thr2) break;
      const double rz = Sm.precond(r, z, y0, ya, yb);
      const double be = rz / rho;
      record(k - 1, 2, be);
      rho = rz;
      for (int e = tid; e < nel; e += kSmallThreads) p[e] = fma(be, p[e], z[e]);
      __syncthreads();
    }
  }
  __syncthreads();
  for (int e = tid; e < nel; e += kSmallThreads) P.x[e] = x[e];
  if (tid == 0) {
    *P.iters = it;
    *P.status = status;
    *P.outer = 0;
    *P.resid = status == kErrBreakdown ? errv : (nb > 0 ? sqrt(rr) / nb : 0.0);
    *P.errval = errv;
  }
}

}  // namespace bt

// Whether an instance of this shape fits the engine (shared memory).
extern "C" int bt_small_fits(int N, int n, int bs64) {
  return N >= 1 && n >= 1 && bt::small_bytes(N, n, bs64) <= bt::kSmallMaxBytes;
}

extern "C" cudaError_t bt_small_launch(const double* const* blk64, int N, int n, int bs64, int m, const double* alpha,
                                       const double* b, double* x, int use_x0, double tol, int maxit,
                                       long long budget, double* hist, int hist_len, int* iters, int* status,
                                       int* outer, double* resid, double* errval, cudaStream_t st) {
  bt::SmallParams P{};
  P.D = blk64[0]; P.O = blk64[1]; P.Dinv = blk64[2]; P.E = blk64[3];
  P.Hd = blk64[4]; P.Hu = blk64[5]; P.Hl = blk64[6];
  P.N = N; P.n = n; P.bs = bs64; P.m = m;
  for (int j = 0; j < bt::kMaxM; ++j) P.alpha[j] = j < m ? alpha[j] : 0.0;
  P.b = b; P.x = x; P.use_x0 = use_x0; P.tol = tol; P.maxit = maxit; P.budget = budget;
  P.hist = hist; P.hist_len = hist_len;
  P.iters = iters; P.status = status; P.outer = outer; P.resid = resid; P.errval = errval;
  const int smem = (int)bt::small_bytes(N, n, bs64);
  cudaError_t e = cudaFuncSetAttribute(bt::bt_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  bt::bt_small_kernel<<<1, bt::kSmallThreads, smem, st>>>(P);
  return cudaGetLastError();
}
