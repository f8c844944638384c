// Small single instances (float64): the whole PCG of one instance in one CTA,
// or in one thread-block cluster of C CTAs, with every block resident in
// shared memory.
//
// For an instance as small as N = 16 block rows of n = 6 (the seven float64
// block arrays D, O, D^-1, E, Hd, Hu, Hl take 32 KB) the persistent kernel's
// bulk-copy pipeline costs more than the arithmetic: each sweep is one chunk,
// each chunk waits for its copy.  Here the blocks are loaded once per solve
// and every iteration runs from shared memory: block-tridiagonal SpMV
// (Eq. 1), the preconditioner apply y0 = G r, y_j = H y_{j-1},
// z = sum_j alpha_j y_j (Sec. 4.1-4.2 closed form), textbook PCG on the
// float64 user vectors with a fixed-order reduction for the dots.
//
// A larger instance (LQR N = 128, n = 12: 1.1 MB of float64 blocks) splits
// its block rows over a cluster of C CTAs (rows [c N / C, (c + 1) N / C) in
// CTA c, at least two rows each): each CTA holds the blocks of its rows (and
// the two rows above, whose O, E, Hl its rows read) and its rows of every
// vector; the one or two halo rows a sweep reads from a neighbour come from
// that CTA's shared memory through the cluster's distributed shared memory,
// after a cluster barrier that makes them final.  A dot product sums each
// CTA's total, then the C totals in rank order, so every CTA holds the same
// bitwise result and takes the same decisions.
//
// Results and statuses are those of the persistent kernel's float64 path
// (recursive residual test ||r|| <= tol ||b||, x0 = 0 or the caller's).
#include <cooperative_groups.h>

#include <cstdint>

#include "../../include/bt.h"
#include "bt_common.cuh"
#include "bt_dd.cuh"

namespace cg = cooperative_groups;

namespace bt {

constexpr int kSmallThreads = 256;
constexpr int kSmallMaxBytes = 200 * 1024;  // shared memory one CTA may take
constexpr int kSmallMaxCluster = 8;         // portable cluster size

struct SmallParams {
  const double *D, *O, *Dinv, *E, *Hd, *Hu, *Hl;  // library slots (column-major, stride bs)
  // mixed handles: the float32 slots (stride bs32) of all seven arrays; D, O
  // above are then the float64 copies the refinement residual uses
  const float *D32, *O32, *Dinv32, *E32, *Hd32, *Hu32, *Hl32;
  int bs32;
  double tol_inner;  // mixed: 0 = automatic (as the persistent kernel)
  int max_outer;
  int scal64;        // mixed: divide the inner step scalars in float64 (else float32, as the persistent kernel)
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

// first block row of CTA c of C
__host__ __device__ inline int small_row0(int N, int C, int c) { return (int)((long long)c * N / C); }

// Largest per-CTA row count and block-slot count over the C CTAs (a CTA keeps
// the slots of rows max(0, s - 2) .. e - 1); every CTA uses the same layout.
__host__ __device__ inline void small_extent(int N, int C, int& rows_max, int& slots_max) {
  rows_max = slots_max = 0;
  for (int c = 0; c < C; ++c) {
    const int s = small_row0(N, C, c), e = small_row0(N, C, c + 1);
    const int lo = s >= 2 ? s - 2 : 0;
    rows_max = rows_max > e - s ? rows_max : e - s;
    slots_max = slots_max > e - lo ? slots_max : e - lo;
  }
}

// Shared memory of one CTA: seven block arrays, eight vectors, scratch.
__host__ __device__ inline long long small_bytes(int N, int n, int bs, int C) {
  int rows_max, slots_max;
  small_extent(N, C, rows_max, slots_max);
  return (7ll * slots_max * bs + 8ll * rows_max * n) * 8 + 64 * 8;
}

// Mixed handles: float64 D, O and the float64 solution and refinement
// residual, then the seven float32 block arrays and eight float32 vectors.
__host__ __device__ inline long long small_bytes_mixed(int N, int n, int bs64, int bs32, int C) {
  int rows_max, slots_max;
  small_extent(N, C, rows_max, slots_max);
  return (2ll * slots_max * bs64 + 2ll * rows_max * n + 64) * 8 + (7ll * slots_max * bs32 + 8ll * rows_max * n) * 4;
}

// Whether C CTAs can hold the instance: every CTA two rows at least (the halo
// of the H sweep then sits in the neighbouring CTA), the shared memory cap.
// bs32 > 0: a mixed handle.
__host__ __device__ inline bool small_fits_c(int N, int n, int bs, int C, int bs32 = 0) {
  if (N < 1 || n < 1 || C < 1 || C > kSmallMaxCluster) return false;
  if (C > 1 && N < 2 * C) return false;
  const long long b = bs32 > 0 ? small_bytes_mixed(N, n, bs, bs32, C) : small_bytes(N, n, bs, C);
  return b <= kSmallMaxBytes;
}

// CL: launched as a cluster of C > 1 CTAs (distributed shared memory and
// cluster barriers); else one CTA, with none of that code.
template <bool CL>
struct Small {
  const SmallParams& P;
  double *D, *O, *Dinv, *E, *Hd, *Hu, *Hl;  // local slots: block row i at (i - lo) * bs
  double* vbase;                            // eight vectors of rows_max * n (local rows)
  double* red;                              // [64] scratch: warp sums, totals, cluster slots
  int N, n, bs, tid, C, rank, s, e, lo, nel, rows_max;
  int s_prev, s_next;  // first rows of the neighbouring CTAs
  int rpar = 0;        // parity of the cluster-sum slot

  __device__ Small(const SmallParams& P_, double* sm) : P(P_) {
    N = P.N;
    n = P.n;
    bs = P.bs;
    tid = threadIdx.x;
    C = 1;
    rank = 0;
    if constexpr (CL) {
      C = (int)cg::this_cluster().num_blocks();
      rank = (int)cg::this_cluster().block_rank();
    }
    s = small_row0(N, C, rank);
    e = small_row0(N, C, rank + 1);
    s_prev = rank > 0 ? small_row0(N, C, rank - 1) : 0;
    s_next = e;
    lo = s >= 2 ? s - 2 : 0;
    nel = (e - s) * n;
    int slots_max;
    small_extent(N, C, rows_max, slots_max);
    const long long A = (long long)slots_max * bs;
    D = sm; O = D + A; Dinv = O + A; E = Dinv + A; Hd = E + A; Hu = Hd + A; Hl = Hu + A;
    vbase = Hl + A;
    red = vbase + 8ll * rows_max * n;
  }
  __device__ double* vec(int k) { return vbase + (long long)k * rows_max * n; }

  // row r (0 <= r < N) of vector v: local, or a neighbour's (same offsets in
  // every CTA of the cluster)
  template <typename T>
  __device__ const T* row(const T* v, int r) {
    if constexpr (CL) {
      if (r < s || r >= e) {
        T* w = const_cast<T*>(v);
        if (r < s) return cg::this_cluster().map_shared_rank(w, rank - 1) + (long long)(r - s_prev) * n;
        return cg::this_cluster().map_shared_rank(w, rank + 1) + (long long)(r - s_next) * n;
      }
    }
    return v + (long long)(r - s) * n;
  }

  // every CTA's writes before it are visible to the whole cluster after it
  __device__ void csync() {
    if constexpr (CL) cg::this_cluster().sync();
    else __syncthreads();
  }

  // Float64 cost model of this engine: on this part a float64 warp
  // instruction costs the SM about the same time whatever the number of its
  // active lanes and whichever warps issue it (measured: the sweeps run no
  // faster with the elements spread over four warps instead of three), so
  // the sums and step scalars below are built from the fewest float64
  // instructions, on as few warps as possible.
  //
  // Totals of the CTA (thread 0's w[q]) -> over the cluster in rank order
  // (the same bits in every CTA) -> post(red) on thread 0 once the totals are
  // in red[16 .. 16 + K), before the barrier that publishes them: the step
  // scalars are formed there, by one thread, and read by the others from
  // red[26 ..).
  template <int K, class Post>
  __device__ void finishK(const double (&w)[K], double (&v)[K], Post post) {
    if (tid == 0) {
#pragma unroll
      for (int q = 0; q < K; ++q) {
        red[16 + q] = w[q];
        red[20 + 2 * rpar + q] = w[q];  // this CTA's totals for the cluster sum
      }
      if constexpr (!CL) post(red);
    }
    if constexpr (CL) {
      cg::this_cluster().sync();
      if (tid < 32) {  // lane c reads CTA c's totals (one remote load each), then a fixed tree
        double t[K];
#pragma unroll
        for (int q = 0; q < K; ++q) t[q] = 0.0;
        if (tid < C) {
          const double* rc = cg::this_cluster().map_shared_rank(red, tid);
#pragma unroll
          for (int q = 0; q < K; ++q) t[q] = rc[20 + 2 * rpar + q];
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1)  // C <= 8; levels over lanes >= C only add zeros
          if (o < C)
#pragma unroll
            for (int q = 0; q < K; ++q) t[q] += __shfl_xor_sync(0xffffffffu, t[q], o);
        if (tid == 0) {
#pragma unroll
          for (int q = 0; q < K; ++q) red[16 + q] = t[q];
          post(red);  // every CTA's thread 0 on the same totals: the same decisions
        }
      }
    }
    // a CTA's slot of parity p is rewritten two sums later, after the next
    // sum's cluster barrier: every CTA has read it by then
    rpar ^= 1;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < K; ++q) v[q] = red[16 + q];
  }

  // v[0..K) (one partial per thread) summed over the CTA (shuffle tree in
  // each warp with elements, then over those warps) and over the cluster.
  template <int K, class Post>
  __device__ void reduceK(double (&v)[K], Post post) {
    // warps past the CTA's elements hold exact zeros: no float64 adds for them
    if ((tid & ~31) < nel) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < K; ++q) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    }
    __syncthreads();  // scratch free (the previous totals and scalars were read)
    if ((tid & 31) == 0)
#pragma unroll
      for (int q = 0; q < K; ++q) red[8 * q + (tid >> 5)] = v[q];
    __syncthreads();
    double w[K];
    if (tid < 32) {
      const int aw = (nel + 31) >> 5;  // warps holding elements; the others' sums are zeros
#pragma unroll
      for (int q = 0; q < K; ++q) w[q] = tid < kSmallThreads / 32 ? red[8 * q + tid] : 0.0;
#pragma unroll
      for (int o = kSmallThreads / 64; o > 0; o >>= 1)
        if (o < aw)  // a level that would only add zeros is skipped (the same bits)
#pragma unroll
          for (int q = 0; q < K; ++q) w[q] += __shfl_xor_sync(0xffffffffu, w[q], o);
    }
    finishK<K>(w, v, post);
  }

  // v[q] + sum over the CTA's elements of a[q][el] b[q][el] (a[q] null: v[q]
  // alone; v[q] is taken from thread 0), then over the cluster and post() as
  // above.  All on warp 0: lane l forms the float64 products of elements
  // l, l + 32, ... in one fma chain, then a shuffle tree -- for 96 elements
  // 3 + 5 float64 instructions per sum instead of 1 + 5 on each of three
  // warps and a tree over the warps.
  //
  // Float32 vectors (the mixed kernel): the same on the float32 pipe, every
  // product split exactly (x y = p + e, e = fma(x, y, -p)) and summed as a
  // double-float pair (error-free two_sum of the high parts, the low parts
  // and rounding errors summed in float32: within about nel 2^-48 of the
  // exact sum), merged into float64 once by lane 0.
  template <int K, typename T, class Post>
  __device__ void dotK(const T* const (&a)[K], const T* const (&b)[K], double (&v)[K], Post post) {
    __syncthreads();  // the vectors are final in this CTA; the previous scalars were read
    double w[K];
    if (tid < 32) {
      if constexpr (sizeof(T) == 8) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
          w[q] = tid == 0 ? v[q] : 0.0;
          if (a[q])
            for (int el = tid; el < nel; el += 32) w[q] = fma(a[q][el], b[q][el], w[q]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
          if (o < nel)  // lanes >= nel hold zeros (no level for them)
#pragma unroll
            for (int q = 0; q < K; ++q)
              if (a[q]) w[q] += __shfl_xor_sync(0xffffffffu, w[q], o);
      } else {
#pragma unroll
        for (int q = 0; q < K; ++q) {
          w[q] = tid == 0 ? v[q] : 0.0;
          if (!a[q]) continue;
          dd acc = dd_make(0.f, 0.f);
          for (int el = tid; el < nel; el += 32) {
            const float x = a[q][el], y = b[q][el];
            const float pr = __fmul_rn(x, y);
            const float er = __fmaf_rn(x, y, -pr);
            const dd t = two_sum(acc.h, pr);
            acc = dd_make(t.h, __fadd_rn(acc.l, __fadd_rn(t.l, er)));
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1)
            if (o < nel)
              acc = dd_add(acc, dd_make(__shfl_xor_sync(0xffffffffu, acc.h, o), __shfl_xor_sync(0xffffffffu, acc.l, o)));
          if (tid == 0) w[q] += f2d_exact(acc.h) + f2d_exact(acc.l);
        }
      }
    }
    finishK<K>(w, v, post);
  }
  template <int K>
  __device__ void reduceK(double (&v)[K]) {
    reduceK<K>(v, [](double*) {});
  }
  __device__ void reduce2(double a, double b, double& ra, double& rb) {
    double v[2] = {a, b};
    reduceK<2>(v);
    ra = v[0];
    rb = v[1];
  }
  __device__ double reduce(double a) {
    double v[1] = {a};
    reduceK<1>(v);
    return v[0];
  }

  // out = (block row of M) v for this CTA's elements (i, a); kind 0: S, 1: G,
  // 2: H; blk = D, O, D^-1, E, Hd, Hu, Hl local slots of stride `sb` (block row
  // i at (i - lo) sb), element type T, accumulation in T
  template <typename T>
  __device__ void sweepT(int kind, const T* const* blk, int sb, const T* v, T* out) {
    const auto slotT = [&](int k, int i) { return blk[k] + (long long)(i - lo) * sb; };
    for (int el = tid; el < nel; el += kSmallThreads) {
      const int li = el / n, a = el - li * n;
      const int i = s + li;
      const T* vi = v + (long long)li * n;
      T acc = T(0);
      const T* M0 = slotT(kind == 0 ? 0 : (kind == 1 ? 2 : 4), i);
      for (int c = 0; c < n; ++c) acc = fma(M0[c * n + a], vi[c], acc);
      if (kind == 0 || kind == 1) {
        // one fma chain over the three blocks (the fewest float64
        // instructions); G's off-diagonal blocks are -E_i, -E_{i-1}^T
        const int km = kind == 0 ? 1 : 3;
        if (i + 1 < N) {  // (i, i+1): O_i / E_i
          const T* Mi = slotT(km, i);
          const T* vn = row(v, i + 1);
          if (kind == 0)
            for (int c = 0; c < n; ++c) acc = fma(Mi[c * n + a], vn[c], acc);
          else
            for (int c = 0; c < n; ++c) acc = fma(-Mi[c * n + a], vn[c], acc);
        }
        if (i >= 1) {  // (i, i-1): O_{i-1}^T / E_{i-1}^T
          const T* Mp = slotT(km, i - 1);
          const T* vp = row(v, i - 1);
          if (kind == 0)
            for (int c = 0; c < n; ++c) acc = fma(Mp[a * n + c], vp[c], acc);
          else
            for (int c = 0; c < n; ++c) acc = fma(-Mp[a * n + c], vp[c], acc);
        }
      } else {
        if (i + 2 < N) {  // (i, i+2): Hu_i
          const T* Mi = slotT(5, i);
          const T* vn = row(v, i + 2);
          for (int c = 0; c < n; ++c) acc = fma(Mi[c * n + a], vn[c], acc);
        }
        if (i >= 2) {  // (i, i-2): Hl_{i-2}
          const T* Mp = slotT(6, i - 2);
          const T* vp = row(v, i - 2);
          for (int c = 0; c < n; ++c) acc = fma(Mp[c * n + a], vp[c], acc);
        }
      }
      out[el] = acc;
    }
  }
  __device__ void sweep(int kind, const double* v, double* out) {
    const double* const blk[7] = {D, O, Dinv, E, Hd, Hu, Hl};
    sweepT<double>(kind, blk, bs, v, out);
  }

  // z = M^-1 r (y0 = G r, y_j = H y_{j-1}, z = y0 + sum_{j>0} alpha_j y_j);
  // returns r . z (products and sum in float64).  r must be final in every CTA
  // (a cluster barrier since its last write).
  template <typename T>
  __device__ double precondT(const T* const* blk, int sb, const T* r, T* z, T* y0, T* ya, T* yb) {
    sweepT<T>(1, blk, sb, r, P.m == 1 ? z : y0);
    if (P.m > 1) {
      const T* yin = y0;
      for (int j = 1; j < P.m; ++j) {
        csync();  // yin final in every CTA (the H sweep reads two rows of the neighbours)
        T* yout = (j & 1) ? ya : yb;
        sweepT<T>(2, blk, sb, yin, yout);
        yin = yout;
        const T aj = (T)P.alpha[j];
        for (int el = tid; el < nel; el += kSmallThreads) z[el] = fma(aj, yout[el], j == 1 ? y0[el] : z[el]);
      }
    }
    double t = 0.0;
    for (int el = tid; el < nel; el += kSmallThreads) t = fma((double)r[el], (double)z[el], t);
    return reduce(t);
  }
  // The same, with r . r summed beside r . z: one sum per iteration fewer
  // when the convergence test waits for the preconditioner (the z of the
  // last iteration is then formed and not used).  post: as in finishK, on the
  // totals (r . z, r . r).
  template <typename T, class Post>
  __device__ double precond2T(const T* const* blk, int sb, const T* r, T* z, T* y0, T* ya, T* yb, double& rr,
                              Post post) {
    sweepT<T>(1, blk, sb, r, P.m == 1 ? z : y0);
    if (P.m > 1) {
      const T* yin = y0;
      for (int j = 1; j < P.m; ++j) {
        csync();
        T* yout = (j & 1) ? ya : yb;
        sweepT<T>(2, blk, sb, yin, yout);
        yin = yout;
        const T aj = (T)P.alpha[j];
        for (int el = tid; el < nel; el += kSmallThreads) z[el] = fma(aj, yout[el], j == 1 ? y0[el] : z[el]);
      }
    }
    const T* const a[2] = {r, r};
    const T* const b[2] = {z, r};
    double v[2] = {0.0, 0.0};
    dotK<2, T>(a, b, v, post);
    rr = v[1];
    return v[0];
  }
  __device__ double precond(const double* r, double* z, double* y0, double* ya, double* yb) {
    const double* const blk[7] = {D, O, Dinv, E, Hd, Hu, Hl};
    return precondT<double>(blk, bs, r, z, y0, ya, yb);
  }
};

template <bool CL>
__global__ void __launch_bounds__(kSmallThreads, 1) bt_small_kernel(const __grid_constant__ SmallParams P) {
  extern __shared__ __align__(16) double smd[];
  Small<CL> Sm(P, smd);
  const int tid = threadIdx.x;
  const long long deadline = clock64() + P.budget;
  // load the blocks of this CTA's rows (and the two rows above) once
  {
    const long long off = (long long)Sm.lo * P.bs, cnt = (long long)(Sm.e - Sm.lo) * P.bs;
    const double* src[7] = {P.D, P.O, P.Dinv, P.E, P.Hd, P.Hu, P.Hl};
    double* dst[7] = {Sm.D, Sm.O, Sm.Dinv, Sm.E, Sm.Hd, Sm.Hu, Sm.Hl};
    const int na = P.m > 1 ? 7 : 4;
    for (int k = 0; k < na; ++k)
      for (long long t = tid; t < cnt; t += kSmallThreads) dst[k][t] = __ldg(src[k] + off + t);
  }
  const int nel = Sm.nel;
  const long long g0 = (long long)Sm.s * P.n;  // this CTA's first element in the user vectors
  double* x = Sm.vec(0);
  double* r = Sm.vec(1);
  double* p = Sm.vec(2);
  double* q = Sm.vec(3);
  double* z = Sm.vec(4);
  double* y0 = Sm.vec(5);
  double* ya = Sm.vec(6);
  double* yb = Sm.vec(7);
  double* const hist = (P.hist && tid == 0 && Sm.rank == 0) ? P.hist : nullptr;
  auto record = [&](int idx, int field, double v) {
    if (hist && idx >= 0 && idx < P.hist_len) hist[(size_t)idx * 3 + field] = v;
  };
  // r0 = b - S x0 (or b with x0 = 0)
  double bb = 0.0;
  for (int el = tid; el < nel; el += kSmallThreads) {
    const double bv = P.b[g0 + el];
    bb = fma(bv, bv, bb);
    x[el] = P.use_x0 ? P.x[g0 + el] : 0.0;
    r[el] = bv;
  }
  Sm.csync();  // x final in every CTA
  if (P.use_x0) {
    Sm.sweep(0, x, q);
    for (int el = tid; el < nel; el += kSmallThreads) r[el] -= q[el];
  }
  double rr_loc = 0.0;
  for (int el = tid; el < nel; el += kSmallThreads) rr_loc = fma(r[el], r[el], rr_loc);
  double bbt, rr;
  Sm.reduce2(bb, rr_loc, bbt, rr);  // also makes r final in every CTA
  const double nb = sqrt(bbt);
  int status = kOK, it = 0;
  double errv = 0.0;
  const double nrhs = P.use_x0 ? nb : sqrt(rr);
  const double thr2 = (P.tol * nrhs) * (P.tol * nrhs);
  if (!isfinite(rr) || !isfinite(nb)) {
    status = kErrNonfinite;
  } else if (nrhs > 0.0 && !(rr <= thr2)) {
    double rho = Sm.precond(r, z, y0, ya, yb);
    for (int el = tid; el < nel; el += kSmallThreads) p[el] = z[el];
    for (int k = 1;; ++k) {
      if (k > P.maxit) {
        status = kErrNoConv;
        it = P.maxit;
        break;
      }
      Sm.csync();  // p final in every CTA
      Sm.sweep(0, p, q);
      // p.q; thread 0 checks it and the cycle budget (rank 0's clock decides
      // for a cluster, through the sum) and divides alpha = rho / p.q
      double pq;
      {
        constexpr int K = CL ? 2 : 1;
        double v[K];
        const double* a[K];
        const double* b[K];
        v[0] = 0.0;
        a[0] = p;
        b[0] = q;
        if constexpr (CL) {
          v[K - 1] = (tid == 0 && Sm.rank == 0 && clock64() > deadline) ? 1.0 : 0.0;
          a[K - 1] = b[K - 1] = nullptr;
        }
        Sm.template dotK<K, double>(a, b, v, [&](double* rd) {
          const double pqv = rd[16];
          bool late;
          if constexpr (CL) late = rd[16 + K - 1] > 0.0;
          else late = clock64() > deadline;
          const int c = late ? kErrTimeout : (!isfinite(pqv) ? kErrNonfinite : (!(pqv > 0.0) ? kErrBreakdown : kOK));
          rd[26] = c == kOK ? rho / pqv : 0.0;
          reinterpret_cast<int*>(rd + 28)[0] = c;
        });
        pq = v[0];
      }
      const int c_pq = reinterpret_cast<const int*>(Sm.red + 28)[0];
      if (c_pq != kOK) {
        status = c_pq;
        it = k - 1;
        if (c_pq == kErrBreakdown) errv = pq;
        break;
      }
      const double al = Sm.red[26];
      if (hist) {
        record(k - 1, 1, al);
        record(k - 1, 2, 0.0);
      }
      for (int el = tid; el < nel; el += kSmallThreads) {
        x[el] = fma(al, p[el], x[el]);
        r[el] = fma(-al, q[el], r[el]);
      }
      Sm.csync();  // r final in every CTA (the G sweep reads neighbouring rows)
      const double* const blk64[7] = {Sm.D, Sm.O, Sm.Dinv, Sm.E, Sm.Hd, Sm.Hu, Sm.Hl};
      // r.z and r.r; thread 0 tests r.r and divides beta = r.z / rho
      const double rz = Sm.template precond2T<double>(blk64, P.bs, r, z, y0, ya, yb, rr, [&](double* rd) {
        const double rzv = rd[16], rrv = rd[17];
        const int c = !isfinite(rrv) ? 1 : (rrv <= thr2 ? 2 : 0);
        rd[27] = c == 0 ? rzv / rho : 0.0;
        reinterpret_cast<int*>(rd + 28)[1] = c;
      });
      it = k;
      if (hist) record(k - 1, 0, sqrt(rr) / nrhs);
      const int c_rr = reinterpret_cast<const int*>(Sm.red + 28)[1];
      if (c_rr == 1) {
        status = kErrNonfinite;
        break;
      }
      if (c_rr == 2) break;
      const double be = Sm.red[27];
      if (hist) record(k - 1, 2, be);
      rho = rz;
      for (int el = tid; el < nel; el += kSmallThreads) p[el] = fma(be, p[el], z[el]);
    }
  }
  for (int el = tid; el < nel; el += kSmallThreads) P.x[g0 + el] = x[el];
  if (tid == 0 && Sm.rank == 0) {
    *P.iters = it;
    *P.status = status;
    *P.outer = 0;
    *P.resid = status == kErrBreakdown ? errv : (nb > 0 ? sqrt(rr) / nb : 0.0);
    *P.errval = errv;
  }
  // no CTA leaves while a neighbour may still read its shared memory
  Sm.csync();
}

// Mixed handles: float32 PCG inside float64 iterative refinement, with the
// persistent kernel's outer rules -- r64 = b - S x in float64 (D, O in
// float64), stop when ||r64|| <= tol ||b||, else an inner float32 PCG on
// r64 / ||r64|| to the inner tolerance (the caller's, else sqrt(tol) in
// [1e-6, 1e-4], loosened to what the remaining factor needs), x += ||r64|| d.
// The dots are summed in float64; the inner step scalars are divided in
// float32 (their float32 use) unless the strict float64 split asks for float64.
template <bool CL>
__global__ void __launch_bounds__(kSmallThreads, 1) bt_small_mixed_kernel(const __grid_constant__ SmallParams P) {
  extern __shared__ __align__(16) double smd[];
  Small<CL> Sm(P, smd);
  const int tid = threadIdx.x, n = P.n;
  const long long deadline = clock64() + P.budget;
  int rows_max, slots_max;
  small_extent(P.N, Sm.C, rows_max, slots_max);
  const long long A64 = (long long)slots_max * P.bs, A32 = (long long)slots_max * P.bs32;
  const long long V = (long long)rows_max * n;
  double* D64 = smd;
  double* O64 = D64 + A64;
  double* x = O64 + A64;  // the float64 solution (this CTA's rows)
  double* r64 = x + V;    // the refinement residual
  Sm.red = r64 + V;       // [64]
  float* f = reinterpret_cast<float*>(Sm.red + 64);
  float* blk32[7];
  for (int k = 0; k < 7; ++k) blk32[k] = f + k * A32;
  float* fv = f + 7 * A32;
  float* xin = fv;
  float* r = fv + V;
  float* p = fv + 2 * V;
  float* q = fv + 3 * V;
  float* z = fv + 4 * V;
  float* y0 = fv + 5 * V;
  float* ya = fv + 6 * V;
  float* yb = fv + 7 * V;
  {
    const long long o64 = (long long)Sm.lo * P.bs, c64 = (long long)(Sm.e - Sm.lo) * P.bs;
    const long long o32 = (long long)Sm.lo * P.bs32, c32 = (long long)(Sm.e - Sm.lo) * P.bs32;
    for (long long t = tid; t < c64; t += kSmallThreads) {
      D64[t] = __ldg(P.D + o64 + t);
      O64[t] = __ldg(P.O + o64 + t);
    }
    const float* src[7] = {P.D32, P.O32, P.Dinv32, P.E32, P.Hd32, P.Hu32, P.Hl32};
    const int na = P.m > 1 ? 7 : 4;
    for (int k = 0; k < na; ++k)
      for (long long t = tid; t < c32; t += kSmallThreads) blk32[k][t] = __ldg(src[k] + o32 + t);
  }
  const double* const blk64[7] = {D64, O64, nullptr, nullptr, nullptr, nullptr, nullptr};
  const float* const cblk32[7] = {blk32[0], blk32[1], blk32[2], blk32[3], blk32[4], blk32[5], blk32[6]};
  const int nel = Sm.nel;
  const long long g0 = (long long)Sm.s * n;
  double* const hist = (P.hist && tid == 0 && Sm.rank == 0) ? P.hist : nullptr;
  auto record = [&](int idx, int field, double v) {
    if (hist && idx >= 0 && idx < P.hist_len) hist[(size_t)idx * 3 + field] = v;
  };
  double bb = 0.0;
  for (int el = tid; el < nel; el += kSmallThreads) {
    const double bv = P.b[g0 + el];
    bb = fma(bv, bv, bb);
    x[el] = P.use_x0 ? P.x[g0 + el] : 0.0;
  }
  const double nb = sqrt(Sm.reduce(bb));  // also makes x final in every CTA
  int status = kOK, iters = 0, outer = 0;
  double resid = 0.0, errv = 0.0;
  if (!isfinite(nb)) {
    status = kErrNonfinite;
  } else if (nb == 0.0) {
    for (int el = tid; el < nel; el += kSmallThreads) x[el] = 0.0;
  } else {
    double nr = nb;
    for (outer = 0;; ++outer) {
      const bool have_r64 = outer > 0 || P.use_x0;
      if (have_r64) {
        Sm.template sweepT<double>(0, blk64, P.bs, x, r64);
        double t = 0.0;
        for (int el = tid; el < nel; el += kSmallThreads) {
          const double rv = P.b[g0 + el] - r64[el];
          r64[el] = rv;
          t = fma(rv, rv, t);
        }
        nr = sqrt(Sm.reduce(t));
        if (!isfinite(nr)) {
          status = kErrNonfinite;
          break;
        }
      }
      resid = nr / nb;
      if (nr <= P.tol * nb) {
        status = kOK;
        break;
      }
      if (outer >= P.max_outer || iters >= P.maxit) {
        status = kErrNoConv;
        break;
      }
      double t_in = P.tol_inner > 0.0 ? P.tol_inner : fmin(1e-4, fmax(1e-6, sqrt(P.tol)));
      const double need = 0.5 * P.tol * nb / nr;
      if (need > t_in) t_in = need;
      if (t_in > 0.5) t_in = 0.5;
      // inner float32 PCG on S d = rhs / nr from d = 0
      const double scale = 1.0 / nr;
      double t = 0.0;
      for (int el = tid; el < nel; el += kSmallThreads) {
        const float rv = (float)((have_r64 ? r64[el] : P.b[g0 + el]) * scale);
        r[el] = rv;
        xin[el] = 0.f;
        t = fma((double)rv, (double)rv, t);
      }
      const double rr0 = Sm.reduce(t);  // also makes r final in every CTA
      const double thr2 = t_in * t_in * rr0;
      const int maxit_in = P.maxit - iters;
      int it = 0, ist = kOK;
      double rr = rr0;
      if (rr0 > 0.0 && !(rr0 <= thr2)) {
        double rho = Sm.template precondT<float>(cblk32, P.bs32, r, z, y0, ya, yb);
        for (int el = tid; el < nel; el += kSmallThreads) p[el] = z[el];
        for (int k = 1;; ++k) {
          if (k > maxit_in) {
            ist = kErrNoConv;
            it = maxit_in;
            break;
          }
          Sm.csync();  // p final in every CTA
          Sm.template sweepT<float>(0, cblk32, P.bs32, p, q);
          // p.q (float64 products and sums); thread 0: the checks and alpha
          // (as in the float64 kernel)
          double pq;
          {
            constexpr int K = CL ? 2 : 1;
            double v[K];
            const float* a[K];
            const float* b[K];
            v[0] = 0.0;
            a[0] = p;
            b[0] = q;
            if constexpr (CL) {
              v[K - 1] = (tid == 0 && Sm.rank == 0 && clock64() > deadline) ? 1.0 : 0.0;
              a[K - 1] = b[K - 1] = nullptr;
            }
            Sm.template dotK<K, float>(a, b, v, [&](double* rd) {
              const double pqv = rd[16];
              bool late;
              if constexpr (CL) late = rd[16 + K - 1] > 0.0;
              else late = clock64() > deadline;
              const int c = late ? kErrTimeout : (!isfinite(pqv) ? kErrNonfinite : (!(pqv > 0.0) ? kErrBreakdown : kOK));
              rd[26] = c != kOK ? 0.0 : (P.scal64 ? rho / pqv : (double)__fdiv_rn((float)rho, (float)pqv));
              reinterpret_cast<int*>(rd + 28)[0] = c;
            });
            pq = v[0];
          }
          const int c_pq = reinterpret_cast<const int*>(Sm.red + 28)[0];
          if (c_pq != kOK) {
            ist = c_pq;
            it = k - 1;
            if (c_pq == kErrBreakdown) errv = pq;
            break;
          }
          const double al = Sm.red[26];
          const float alf = (float)al;
          if (hist) {
            record(iters + k - 1, 1, al);
            record(iters + k - 1, 2, 0.0);
          }
          for (int el = tid; el < nel; el += kSmallThreads) {
            xin[el] = fmaf(alf, p[el], xin[el]);
            r[el] = fmaf(-alf, q[el], r[el]);
          }
          Sm.csync();  // r final in every CTA (the G sweep reads neighbouring rows)
          // r.z and r.r; thread 0 tests r.r and divides beta
          const double rz = Sm.template precond2T<float>(cblk32, P.bs32, r, z, y0, ya, yb, rr, [&](double* rd) {
            const double rzv = rd[16], rrv = rd[17];
            const int c = !isfinite(rrv) ? 1 : (rrv <= thr2 ? 2 : 0);
            rd[27] = c != 0 ? 0.0 : (P.scal64 ? rzv / rho : (double)__fdiv_rn((float)rzv, (float)rho));
            reinterpret_cast<int*>(rd + 28)[1] = c;
          });
          it = k;
          if (hist) record(iters + k - 1, 0, sqrt(rr / rr0));
          const int c_rr = reinterpret_cast<const int*>(Sm.red + 28)[1];
          if (c_rr == 1) {
            ist = kErrNonfinite;
            break;
          }
          if (c_rr == 2) break;
          const double be = Sm.red[27];
          if (hist) record(iters + k - 1, 2, be);
          rho = rz;
          const float bef = (float)be;
          for (int el = tid; el < nel; el += kSmallThreads) p[el] = fmaf(bef, p[el], z[el]);
        }
      }
      iters += it;
      if (ist == kErrBreakdown || ist == kErrNonfinite || ist == kErrTimeout) {
        status = ist;
        break;
      }
      for (int el = tid; el < nel; el += kSmallThreads) x[el] = fma(nr, (double)xin[el], x[el]);
      Sm.csync();  // x final in every CTA before the next residual
    }
  }
  for (int el = tid; el < nel; el += kSmallThreads) P.x[g0 + el] = x[el];
  if (tid == 0 && Sm.rank == 0) {
    *P.iters = iters;
    *P.status = status;
    *P.outer = outer;
    *P.resid = status == kErrBreakdown ? errv : resid;
    *P.errval = errv;
  }
  Sm.csync();  // no CTA leaves while a neighbour may still read its shared memory
}

}  // namespace bt

// The cluster size of the engine for an instance of this shape (bs32 > 0: a
// mixed handle): 1 where one CTA holds it, else the smallest of 2, 4, 8 that
// does; 0 where none does.  want > 0 asks for exactly that size (0 if it does
// not fit).
extern "C" int bt_small_cluster(int N, int n, int bs64, int bs32, int want) {
  if (want > 0) return bt::small_fits_c(N, n, bs64, want, bs32) ? want : 0;
  for (int C = 1; C <= bt::kSmallMaxCluster; C *= 2)
    if (bt::small_fits_c(N, n, bs64, C, bs32)) return C;
  return 0;
}

template <bool MIX>
static cudaError_t small_launch(const bt::SmallParams& P, int smem, int C, cudaStream_t st) {
  if (C == 1) {
    const auto kern = MIX ? bt::bt_small_mixed_kernel<false> : bt::bt_small_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<1, bt::kSmallThreads, smem, st>>>(P);
    return cudaGetLastError();
  }
  const auto kern = MIX ? bt::bt_small_mixed_kernel<true> : bt::bt_small_kernel<true>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)C);
  cfg.blockDim = dim3(bt::kSmallThreads);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kern, P);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// blk64: D, O, D^-1, E, Hd, Hu, Hl float64 slots (stride bs64; a mixed handle
// passes its float64 D, O only) and blk32 the float32 slots (stride bs32) of a
// mixed handle, else null.
extern "C" cudaError_t bt_small_launch(const double* const* blk64, const float* const* blk32, int N, int n, int bs64,
                                       int bs32, int m, const double* alpha, const double* b, double* x, int use_x0,
                                       double tol, double tol_inner, int max_outer, int maxit, long long budget,
                                       double* hist, int hist_len, int* iters, int* status, int* outer,
                                       double* resid, double* errval, int scal64, int C, cudaStream_t st) {
  const bool mix = blk32 != nullptr;
  bt::SmallParams P{};
  P.D = blk64[0]; P.O = blk64[1]; P.Dinv = blk64[2]; P.E = blk64[3];
  P.Hd = blk64[4]; P.Hu = blk64[5]; P.Hl = blk64[6];
  if (mix) {
    P.D32 = blk32[0]; P.O32 = blk32[1]; P.Dinv32 = blk32[2]; P.E32 = blk32[3];
    P.Hd32 = blk32[4]; P.Hu32 = blk32[5]; P.Hl32 = blk32[6];
  }
  P.bs32 = bs32;
  P.tol_inner = tol_inner;
  P.max_outer = max_outer;
  P.scal64 = scal64;
  P.N = N; P.n = n; P.bs = bs64; P.m = m;
  for (int j = 0; j < bt::kMaxM; ++j) P.alpha[j] = j < m ? alpha[j] : 0.0;
  P.b = b; P.x = x; P.use_x0 = use_x0; P.tol = tol; P.maxit = maxit; P.budget = budget;
  P.hist = hist; P.hist_len = hist_len;
  P.iters = iters; P.status = status; P.outer = outer; P.resid = resid; P.errval = errval;
  if (!bt::small_fits_c(N, n, bs64, C, mix ? bs32 : 0)) return cudaErrorInvalidValue;
  const int smem = (int)(mix ? bt::small_bytes_mixed(N, n, bs64, bs32, C) : bt::small_bytes(N, n, bs64, C));
  return mix ? small_launch<true>(P, smem, C, st) : small_launch<false>(P, smem, C, st);
}
