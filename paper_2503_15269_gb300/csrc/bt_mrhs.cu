// Many right-hand sides: J = 64 independent PCG recurrences on one SPD
// block-tridiagonal matrix, sharing every block sweep (the block products
// become n x n by n x J contractions).  Float32 inner PCG inside float64
// iterative refinement, the optimal-parameter preconditioner of Sec. 3-4
// (a = 1, polynomial coefficients alpha), textbook PCG per column.
//
// One cooperative launch; G CTAs split the block rows.  Rows are processed
// in gather form, so every output row is independent (no carries between
// CTAs):
//   A   Q_i  = D_i P_i + O_i P_{i+1} + O_{i-1}^T P_{i-1}                 (Eq. 1)
//   B1  Y0_i = D_i^-1 R_i - E_i R_{i+1} - E_{i-1}^T R_{i-1}              (Sec. 4.1)
//   B2  Yj_i = Hd_i Y_i + Hu_i Y_{i+2} + Hl_{i-2} Y_{i-2},  Z += alpha_j Yj (Sec. 4.2)
// with per-column scalars alpha_j, beta_j, rho_j and a per-column active mask;
// grid barriers (bounded) separate the phases.  Vectors are [N][n][J]
// (block row i, then its n rows, then the J columns), J = 64.
//
// The float32 sweeps stage each row job's three blocks in shared memory with
// cp.async (double-buffered: the next row's blocks load while the current
// one computes) and keep the vector rows in a ring of 2k+2 rows, each loaded
// once per sweep.  The block products are register-tiled, 4 rows x 4 columns
// of the output per thread; two thread halves take the two halves of the k
// range of every product (12 warps busy for n = 48, three per scheduler), and
// one half adds the other's partial tile through shared memory before the
// finalize.  The float64 residual sweep (once per refinement step) stages one
// row job at a time.
#include <cstdint>

#include "../../include/bt.h"
#include "bt_common.cuh"

namespace bt {

constexpr int kJ = 64;              // right-hand-side columns per solve
constexpr int kMThreads = 384;
constexpr int kMHalf = 192;         // output tiles one thread half covers (n <= 48 split in k)
constexpr int kMaxNMulti = 64;      // n <= 64: 16 row groups of 4 at most
static_assert(kMaxNMulti / 4 * 16 <= kMThreads, "one pass covers every output tile of the largest block");
constexpr int kVB = 2;              // float4s a thread loads before storing in the vector passes

struct MParams {
  const float *D32, *O32, *Dinv32, *E32, *Hd32, *Hu32, *Hl32;  // library layout (column-major, padded)
  const double *D64, *O64;
  int N, n, bs32, bs64, m;
  float alpha[kMaxM];
  // float64 vectors [N][n][J]
  const double* B64;
  double* X64;
  double* R64;
  // float32 vectors [N][n][J]
  float *Xin, *R, *P, *Q, *Y0, *Ya, *Yb, *Z;
  float* P2;            // second p buffer: the A sweep writes the new p there (n <= 48)
  double* red;          // [2][G][kJ]
  unsigned* bar;
  int* abort_flag;
  double tol, tol_inner;
  int maxit, max_outer;
  long long budget;
  int G;
  int nrhs;
  // results per column
  int* iters;
  int* status;
  double* resid;
  int* outer;
};

__device__ __forceinline__ void cp16(void* smem, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// copy `count` floats (multiple of 4, 16-byte aligned) global -> shared
__device__ __forceinline__ void cp_block(float* dst, const float* src, int count) {
  for (int t = threadIdx.x * 4; t < count; t += kMThreads * 4) cp16(dst + t, src + t);
}
__device__ __forceinline__ void cp_blockd(double* dst, const double* src, int count) {
  for (int t = threadIdx.x * 2; t < count; t += kMThreads * 2) cp16(dst + t, src + t);
}

// 4 consecutive elements from shared memory (16-byte aligned for float,
// two 16-byte loads for double).
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
  const double2 q0 = *reinterpret_cast<const double2*>(p);
  const double2 q1 = *reinterpret_cast<const double2*>(p + 2);
  v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
}

// acc[r][c] (+/-)= sum_{k0 <= k < k1} M(a0+r, k) X(k, j0+c): M column-major
// n x n, X n x J; NEG subtracts (the negation folds into the FMA).
template <bool NEG = false, typename T>
__device__ __forceinline__ void prod_direct(const T* __restrict__ M, const T* __restrict__ X, int n, int a0, int j0,
                                            T acc[4][4], int k0, int k1) {
#pragma unroll 8
  for (int k = k0; k < k1; ++k) {
    T mv[4], xv[4];
    ld4(M + k * n + a0, mv);
    ld4(X + k * kJ + j0, xv);
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = fma(NEG ? -mv[r] : mv[r], xv[c], acc[r][c]);
  }
}

// acc[r][c] (+/-)= sum_{k0 <= k < k1} M(k, a0+r) X(k, j0+c): the transposed
// block (n, k0, k1 multiples of 4).
template <bool NEG = false, typename T>
__device__ __forceinline__ void prod_trans(const T* __restrict__ M, const T* __restrict__ X, int n, int a0, int j0,
                                           T acc[4][4], int k0, int k1) {
#pragma unroll 2
  for (int k = k0; k < k1; k += 4) {
    T mr[4][4], xr[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r) ld4(M + (a0 + r) * n + k, mr[r]);   // M(k..k+3, a0+r)
#pragma unroll
    for (int q = 0; q < 4; ++q) ld4(X + (k + q) * kJ + j0, xr[q]);  // X(k+q, j0..j0+3)
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(NEG ? -mr[r][q] : mr[r][q], xr[q][c], acc[r][c]);
  }
}

struct MSolver {
  const MParams& P;
  char* sm;
  int g, G, N, n, s, e;
  long long deadline;
  int bar_count;
  bool fail;
  double* colbuf;   // smem [kJ] scratch for reduced values
  double* colred;   // smem scratch for the cross-CTA column sums ([kMThreads / kJ][kJ])

  __device__ MSolver(const MParams& P_, char* sm_) : P(P_), sm(sm_) {}

  // Grid barrier with a per-column reduction of v (one value per column,
  // held by threads tid < kJ after an in-CTA reduction).  Bounded.
  __device__ void grid_reduce(double* colv /* smem [kJ], CTA partials in, totals out */) {
    if (fail) return;
    __syncthreads();
    int* flag = reinterpret_cast<int*>(sm);
    const int par = bar_count & 1;  // every thread keeps the barrier count
    ++bar_count;
    if (threadIdx.x < kJ) P.red[((size_t)par * G + g) * kJ + threadIdx.x] = colv[threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();  // after the CTA barrier: publishes every thread's slot store
      atomicAdd(P.bar, 1u);
      const unsigned target = (unsigned)G * (unsigned)bar_count;
      int bad = 0;
      while (ld_acquire_u32(P.bar) < target) {
        if (ld_volatile_i32(P.abort_flag) || clock64() > deadline) {
          bad = 1;
          break;
        }
      }
      if (bad) atomicExch(P.abort_flag, 1);
      flag[0] = bad;
    }
    __syncthreads();
    if (flag[0]) {
      fail = true;
      return;
    }
    // Totals: the kQ x 64 threads each sum a kQ-th of the G slots of one
    // column with independent L2 loads (the barrier above acquired them),
    // then the parts are added in a fixed order (bitwise reproducible).
    {
      constexpr int kQ = kMThreads / kJ;
      static_assert(kMThreads == kQ * kJ, "whole groups of 64 threads");
      double* part = colred;  // [kQ][kJ] doubles of the CTA's scratch
      const int q = threadIdx.x / kJ, j = threadIdx.x % kJ;
      const int g0 = q * G / kQ, g1 = (q + 1) * G / kQ;
      const double* src = P.red + (size_t)par * G * kJ + j;
      double t = 0.0;
#pragma unroll 8
      for (int gg = g0; gg < g1; ++gg) t += __ldcg(src + (size_t)gg * kJ);
      part[q * kJ + j] = t;
      __syncthreads();
      if (threadIdx.x < kJ) {
        double sum = part[j];
#pragma unroll
        for (int qq = 1; qq < kQ; ++qq) sum += part[qq * kJ + j];
        colv[j] = sum;
      }
    }
    __syncthreads();
  }

  __device__ void barrier() {
    double* cv = colbuf;
    if (threadIdx.x < kJ) cv[threadIdx.x] = 0.0;
    grid_reduce(cv);
  }
};

// Element (row, a, j0..j0+3) of an [N][n][kJ] vector: 4 consecutive columns.
__device__ __forceinline__ float4 ldv4(const float* v, size_t idx) { return *reinterpret_cast<const float4*>(v + idx); }
__device__ __forceinline__ void stv4(float* v, size_t idx, float4 x) { *reinterpret_cast<float4*>(v + idx) = x; }
__device__ __forceinline__ void widen(const Accum<float> (&a)[4], double (&d)[4]) {
  for (int c = 0; c < 4; ++c) d[c] = a[c].value();
}

// Reduce per-thread column partials part[jg][4] (threads laid out t = ag*16 + jg)
// into colv[kJ] over the CTA, fixed order.
__device__ __forceinline__ void cta_col_reduce(const double (&pv)[4], double* scratch /* [ngroups][kJ] */,
                                               double* colv, int ngroups) {
  const int t = threadIdx.x;
  const int jg = t & 15, ag = t >> 4;
  if (ag < ngroups)
    for (int c = 0; c < 4; ++c) scratch[ag * kJ + 4 * jg + c] = pv[c];
  __syncthreads();
  if (t < kJ) {
    double s = 0.0;
    for (int a = 0; a < ngroups; ++a) s += scratch[a * kJ + t];
    colv[t] = s;
  }
  __syncthreads();
}

}  // namespace bt

using namespace bt;

// Shared memory layout (bytes):
//   [0, 256)          flags
//   [256, +512)       colA  (double[kJ])   per-column scalars / reductions
//   ... colB, colC, colD, rho, alpha, beta, act, nbv, nrv, tin
//   then scratch [16][kJ] doubles (column partials)
//   then two job buffers of kJobBytes
constexpr int kColBytes = kJ * 8;
constexpr int kMSmScalars = 256;
constexpr int kMNumCols = 13;  // 12 double columns + float alpha/beta copies
constexpr int kMSmScratch = kMSmScalars + kMNumCols * kColBytes;
constexpr int kMSmXch = kMSmScratch + (kMThreads / 16) * kJ * 8;  // float4 [4][kMHalf]
constexpr int kMSmJobs = kMSmXch + 4 * kMHalf * 16;

__host__ __device__ constexpr int mrhs_job_bytes(int n) {
  // float32 job: 3 blocks + 3 vector blocks; float64 job: same in doubles
  return 3 * n * n * 8 + 3 * n * kJ * 8;
}

namespace bt {

enum MPhase : int { MP_A = 0, MP_B1 = 1, MP_B2 = 2 };

// The p update p = z + beta p folded into the A sweep (z null: off).  The
// ring stages the old p; each ring row, once its copy has landed, becomes
// z + beta p in place (z staged beside it), and the owned rows are also
// written to `pout`.  `beta`: the per-column float beta in shared memory.
struct Fold {
  const float* z;
  float* pout;
  const float* beta;
};

// Float32 sweeps: the vector rows a row job reads (i-k, i, i+k) come from a
// ring of 2k+2 rows in shared memory, each loaded once per sweep (one row
// ahead, with the blocks of the next job), instead of three copies per row in
// every job; the ring occupies the room of the second job's vector rows.
//
// Thread t covers output tile u (row group u / 16, column group u % 16) over
// the k range of its half: for n <= 48 the 4n tiles fit one half of the CTA
// and the second half takes k in [kh, n); for larger n one pass covers all
// tiles and k.  The partial tiles of the second half go through `xch`.
// `pre` (may be null): a float32 vector whose tile of the row the finalize
// needs (passed to it as pf, row r of the tile at pf[r * pstride]).  For n <= 48 each thread
// copies its tile into shared memory with cp.async before the products, so
// the load overlaps them; larger blocks leave no room and load it directly.
//
// `fd` (A sweep, n <= 48 only): the p update folded in.  The prologue rows are
// updated by all threads before the first products; every later row by the
// second thread half while the first runs the finalize, between the row's
// two barriers, so that the next row's products see it.  Its z rows use the
// ring's two spare slots (A keeps 4 of 6) and the staged-tile region: three
// slots, row r in slot r % 3.
template <typename Fin, typename Blk>
__device__ void msweep_ring(MSolver& Sv, int phase, const float* v_in, const float* pre, const Fold& fd, Fin fin,
                            Blk blk) {
  const int n = Sv.n, N = Sv.N;
  const int tid = threadIdx.x;
  const int ngroups = n / 4;
  const int ntile = ngroups * 16;
  const bool split = ntile <= kMHalf;
  const int half = split ? tid / kMHalf : 0;
  const int u = split ? tid - half * kMHalf : tid;
  const int jg = u & 15, ag = u >> 4;
  const bool active = u < ntile;
  const int a0 = 4 * ag, j0 = 4 * jg;
  const int kh = split ? 4 * ((ngroups + 1) / 2) : n;
  const int k0 = half ? kh : 0, k1 = half ? n : kh;
  const int bb = n * n, vb = n * kJ;
  const int k = (phase == MP_B2) ? 2 : 1;
  const int kv = 2 * k + 2;
  float* blocks = reinterpret_cast<float*>(Sv.sm + kMSmJobs);  // [2][3 bb]
  float* ring = blocks + 6 * bb;                               // [kv][vb]
  float4* xch = reinterpret_cast<float4*>(Sv.sm + kMSmXch);    // [4][kMHalf] partial tiles
  float4* pstage = reinterpret_cast<float4*>(Sv.sm + kMSmJobs + mrhs_job_bytes(n));  // [4][kMHalf], n <= 48
  const auto slot = [&](int r) { return ring + (size_t)(((r % kv) + kv) % kv) * vb; };
  const bool fold = fd.z != nullptr && split && phase == MP_A;
  const auto zslot = [&](int r) {
    const int j = r % 3;  // r >= 0
    return j < 2 ? ring + (size_t)(4 + j) * vb : reinterpret_cast<float*>(pstage);
  };
  const auto fold_row = [&](int r, int t0, int nt) {  // ring row r := z_r + beta p_r
    float4* ps = reinterpret_cast<float4*>(slot(r));
    const float4* zs = reinterpret_cast<const float4*>(zslot(r));
    const float4* b4 = reinterpret_cast<const float4*>(fd.beta);
    float4* po = reinterpret_cast<float4*>(fd.pout + (size_t)r * vb);
    const bool own = r >= Sv.s && r < Sv.e;
    for (int q = t0; q < vb / 4; q += nt) {
      const float4 b = b4[q & 15], pp = ps[q], zz = zs[q];
      const float4 w = make_float4(fmaf(b.x, pp.x, zz.x), fmaf(b.y, pp.y, zz.y), fmaf(b.z, pp.z, zz.z),
                                   fmaf(b.w, pp.w, zz.w));
      ps[q] = w;
      if (own) po[q] = w;
    }
  };
  const auto issue_blocks = [&](int row, int buf) {
    float* m = blocks + (size_t)buf * 3 * bb;
    cp_block(m, blk(0, row), bb);
    if (row + k < N) cp_block(m + bb, blk(1, row), bb);
    if (row - k >= 0) cp_block(m + 2 * bb, blk(2, row - k), bb);
  };
  const int s = Sv.s, e = Sv.e;
  // prologue: the first job's blocks and vector rows s-k .. s+k
  issue_blocks(s, 0);
  for (int r = max(0, s - k); r <= min(N - 1, s + k); ++r) {
    cp_block(slot(r), v_in + (size_t)r * vb, vb);
    if (fold) cp_block(zslot(r), fd.z + (size_t)r * vb, vb);
  }
  cp_commit();
  if (fold) {  // the prologue rows, before any later copy can reuse their z slots
    cp_wait<0>();
    __syncthreads();
    for (int r = max(0, s - k); r <= min(N - 1, s + k); ++r) fold_row(r, tid, kMThreads);
    __syncthreads();
  }
  for (int row = s; row < e; ++row) {
    const int it = row - s;
    if (row + 1 < e) {  // the next job: its one new vector row, then its blocks (two groups)
      const int nr = row + 1 + k;
      if (nr < N) {
        cp_block(slot(nr), v_in + (size_t)nr * vb, vb);
        if (fold) cp_block(zslot(nr), fd.z + (size_t)nr * vb, vb);
      }
      cp_commit();
      issue_blocks(row + 1, (it + 1) & 1);
      cp_commit();
      cp_wait<2>();  // everything but the two groups just issued
    } else {
      cp_wait<0>();
    }
    __syncthreads();
    const float* m0 = blocks + (size_t)(it & 1) * 3 * bb;
    const float* m1 = m0 + bb;
    const float* m2 = m0 + 2 * bb;
    const float* xc = slot(row);
    if (pre && split) {
      if (half == 0 && active)
#pragma unroll
        for (int r = 0; r < 4; ++r) cp16(pstage + r * kMHalf + u, pre + (size_t)row * vb + (size_t)(a0 + r) * kJ + j0);
      cp_commit();
    }
    // one accumulator: G's off-diagonal blocks enter with a minus sign
    float out[4][4] = {};
    if (active) {
      prod_direct(m0, xc, n, a0, j0, out, k0, k1);
      if (phase == MP_B1) {
        if (row + k < N) prod_direct<true>(m1, slot(row + k), n, a0, j0, out, k0, k1);
        if (row - k >= 0) prod_trans<true>(m2, slot(row - k), n, a0, j0, out, k0, k1);
      } else {
        if (row + k < N) prod_direct(m1, slot(row + k), n, a0, j0, out, k0, k1);
        if (row - k >= 0) {
          if (phase == MP_B2) prod_direct(m2, slot(row - k), n, a0, j0, out, k0, k1);
          else prod_trans(m2, slot(row - k), n, a0, j0, out, k0, k1);
        }
      }
    }
    if (split && half == 1 && active)
#pragma unroll
      for (int r = 0; r < 4; ++r) xch[r * kMHalf + u] = make_float4(out[r][0], out[r][1], out[r][2], out[r][3]);
    if (fold) cp_wait<1>();  // the next row's new ring row (and its z) has landed; its blocks may not
    // After this barrier every product of the row is done: the next row's
    // copies (into the other block buffer and the ring slot of row - k) may
    // start while the finalize still reads this row's ring slot.
    __syncthreads();
    if (fold && half == 1 && row + 1 < e && row + 1 + k < N) fold_row(row + 1 + k, u, kMHalf);
    if (half == 0 && active) {
      if (split)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const float4 q = xch[r * kMHalf + u];
          out[r][0] += q.x; out[r][1] += q.y; out[r][2] += q.z; out[r][3] += q.w;
        }
      // the tile of `pre`: row r of it at pf[r * pstride]
      const float4* pf = nullptr;
      int pstride = 0;
      if (pre) {
        if (split) {
          cp_wait<0>();  // this thread's own tile (and the next row's copies, already under way)
          pf = pstage + u;
          pstride = kMHalf;
        } else {
          pf = reinterpret_cast<const float4*>(pre + (size_t)row * vb + (size_t)a0 * kJ + j0);
          pstride = kJ / 4;
        }
      }
      fin(row, a0, j0, out, xc, pf, pstride);
    }
  }
  __syncthreads();
}

// One float32 sweep (A, B1 or B2) over the owned rows, through the ring.
template <typename Fin>
__device__ void msweep32(MSolver& Sv, int phase, const float* v_in, const float* pre, Fin fin,
                         const Fold& fd = Fold{nullptr, nullptr, nullptr}) {
  const MParams& P = Sv.P;
  if (Sv.e <= Sv.s) return;
  auto blk = [&](int which, int row) -> const float* {
    // which: 0 = first (D, D^-1, Hd), 1 = second (O, E, Hu), 2 = third (O, E, Hl)
    const float* A;
    if (phase == MP_A) A = (which == 0) ? P.D32 : P.O32;
    else if (phase == MP_B1) A = (which == 0) ? P.Dinv32 : P.E32;
    else A = (which == 0) ? P.Hd32 : (which == 1 ? P.Hu32 : P.Hl32);
    return A + (size_t)row * P.bs32;
  };
  msweep_ring(Sv, phase, v_in, pre, fd, fin, blk);
}

// The float64 refinement-residual sweep q = S x (Eq. 1) over the owned rows:
// one job buffer (three float64 blocks and three vector rows) fills the
// region the float32 sweeps double-buffer, so each row's copies complete
// before its products.  It runs once per refinement step.  The finalize
// functor receives the 4x4 tile (rows a0.., columns j0..) of row i.
template <typename Fin>
__device__ void msweep64(MSolver& Sv, const double* v_in, Fin fin) {
  const MParams& P = Sv.P;
  const int n = Sv.n, N = Sv.N;
  const int tid = threadIdx.x;
  const int ngroups = n / 4;
  const int jg = tid & 15, ag = tid >> 4;
  const bool active = ag < ngroups;
  const int a0 = 4 * ag, j0 = 4 * jg;
  const int bb = n * n, vb = n * kJ;
  double* m0 = reinterpret_cast<double*>(Sv.sm + kMSmJobs);  // D_i
  double* m1 = m0 + bb;                                        // O_i
  double* m2 = m0 + 2 * bb;                                    // O_{i-1}
  double* xl = m0 + 3 * bb;                                    // x rows i-1, i, i+1
  double* xc = xl + vb;
  double* xr = xc + vb;
  for (int row = Sv.s; row < Sv.e; ++row) {
    cp_blockd(m0, P.D64 + (size_t)row * P.bs64, bb);
    if (row + 1 < N) cp_blockd(m1, P.O64 + (size_t)row * P.bs64, bb);
    if (row >= 1) cp_blockd(m2, P.O64 + (size_t)(row - 1) * P.bs64, bb);
    for (int d = -1; d <= 1; ++d) {
      const int r = row + d;
      if (r >= 0 && r < N) cp_blockd(xl + (d + 1) * vb, v_in + (size_t)r * vb, vb);
    }
    cp_commit();
    cp_wait<0>();
    __syncthreads();
    double out[4][4] = {};
    if (active) {
      prod_direct(m0, xc, n, a0, j0, out, 0, n);                // D_i x_i
      if (row + 1 < N) prod_direct(m1, xr, n, a0, j0, out, 0, n);  // O_i x_{i+1}
      if (row >= 1) prod_trans(m2, xl, n, a0, j0, out, 0, n);      // O_{i-1}^T x_{i-1}
    }
    if (active) fin(row, a0, j0, out, xc);
    __syncthreads();
  }
}

// The kernel: mixed-precision refinement around float32 PCG, all columns.
__global__ void __launch_bounds__(kMThreads, 1) bt_mrhs_kernel(const __grid_constant__ MParams P) {
  extern __shared__ __align__(128) char smem[];
  MSolver Sv(P, smem);
  Sv.g = blockIdx.x;
  Sv.G = P.G;
  Sv.N = P.N;
  Sv.n = P.n;
  Sv.s = (int)((long long)Sv.g * P.N / P.G);
  Sv.e = (int)((long long)(Sv.g + 1) * P.N / P.G);
  Sv.deadline = clock64() + P.budget;
  Sv.bar_count = 0;
  Sv.fail = false;
  double* col = reinterpret_cast<double*>(smem + kMSmScalars);
  double* colR = col + 0 * kJ;     // reduction buffer
  double* rho = col + 1 * kJ;
  double* alp = col + 2 * kJ;
  double* bet = col + 3 * kJ;
  double* actv = col + 4 * kJ;     // 1 active in the inner solve, 0 frozen
  double* nbv = col + 5 * kJ;      // ||b_j||
  double* nrv = col + 6 * kJ;      // ||r64_j||
  double* tin = col + 7 * kJ;      // inner tolerance per column (squared)
  double* outer_act = col + 8 * kJ;  // 1 while the column needs refinement
  double* itc = col + 9 * kJ;      // inner iterations per column
  double* scl = col + 10 * kJ;     // 1 / ||r64_j||
  double* rrv = col + 11 * kJ;
  float* alpf = reinterpret_cast<float*>(col + 12 * kJ);  // float copies of alpha_j, beta_j
  float* betf = alpf + kJ;
  double* scratch = reinterpret_cast<double*>(smem + kMSmScratch);
  Sv.colbuf = colR;
  Sv.colred = scratch;
  const int n = P.n;
  const int tid = threadIdx.x;
  const int ngroups = n / 4;
  const size_t vb = (size_t)n * kJ;
  const int J = kJ;
  const int m = P.m;
  const bool fold = 4 * n <= kMHalf;  // p update folded into the A sweep (the k-split layout)

  // ||b_j||^2 and x64 = 0 over the owned rows
  {
    double pv[4] = {0, 0, 0, 0};
    const int jg = tid & 15, ag = tid >> 4;
    if (ag < ngroups)
      for (int row = Sv.s; row < Sv.e; ++row)
        for (int r = 0; r < 4; ++r)
          for (int c = 0; c < 4; ++c) {
            const size_t idx = (size_t)row * vb + (size_t)(4 * ag + r) * J + 4 * jg + c;
            const double bv = P.B64[idx];
            pv[c] += bv * bv;
            P.X64[idx] = 0.0;
          }
    cta_col_reduce(pv, scratch, colR, ngroups);
    Sv.grid_reduce(colR);
    if (tid < J) {
      nbv[tid] = sqrt(colR[tid]);
      const bool live = tid < P.nrhs && nbv[tid] > 0.0;
      outer_act[tid] = live ? 1.0 : 0.0;
      itc[tid] = 0.0;
      nrv[tid] = nbv[tid];
    }
    __syncthreads();
  }
  int outer = 0;
  int total_it = 0;
  for (outer = 0; outer <= P.max_outer && !Sv.fail; ++outer) {
    // ---- refinement residual r64 = b - S x64 (float64), skipped at x = 0
    if (outer > 0) {
      double pv[4] = {0, 0, 0, 0};
      msweep64(Sv, P.X64, [&](int row, int a0, int j0, double (&o)[4][4], const double*) {
        for (int r = 0; r < 4; ++r)
          for (int c = 0; c < 4; ++c) {
            const size_t idx = (size_t)row * vb + (size_t)(a0 + r) * J + j0 + c;
            const double rv = P.B64[idx] - o[r][c];
            P.R64[idx] = rv;
            pv[c] += rv * rv;
          }
      });
      cta_col_reduce(pv, scratch, colR, ngroups);
      Sv.grid_reduce(colR);
      if (tid < J) nrv[tid] = sqrt(colR[tid]);
      __syncthreads();
    }
    // convergence of the true residual per column
    if (tid < J) {
      const bool live = outer_act[tid] > 0.0 && !(nrv[tid] <= P.tol * nbv[tid]);
      if (outer_act[tid] > 0.0 && !isfinite(nrv[tid])) outer_act[tid] = -1.0;  // non-finite
      else outer_act[tid] = live ? 1.0 : (outer_act[tid] < 0.0 ? -1.0 : 0.0);
      const bool a = outer_act[tid] > 0.0;
      scl[tid] = a ? 1.0 / nrv[tid] : 0.0;
      double t = P.tol_inner;
      if (a) {
        const double need = 0.5 * P.tol * nbv[tid] / nrv[tid];
        if (need > t) t = need;
        if (t > 0.5) t = 0.5;
      }
      tin[tid] = t * t;
      actv[tid] = a ? 1.0 : 0.0;
    }
    __syncthreads();
    const int any = __syncthreads_or(tid < J && actv[tid] > 0.0);
    if (!any || outer == P.max_outer || total_it >= P.maxit) break;
    // ---- inner float32 PCG: r = rhs, x_in = 0
    {
      const int jg = tid & 15, ag = tid >> 4;
      if (ag < ngroups)
        for (int row = Sv.s; row < Sv.e; ++row)
          for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c) {
              const int j = 4 * jg + c;
              const size_t idx = (size_t)row * vb + (size_t)(4 * ag + r) * J + j;
              const double src = (outer > 0) ? P.R64[idx] : P.B64[idx];
              const float rv = (float)(src * scl[j]);
              P.R[idx] = rv;
              P.Xin[idx] = 0.0f;
            }
      Sv.barrier();
    }
    // z0 = M^-1 r0 ; rho = r.z
    auto apply_precond = [&](double* rzout) {
      // r.z per column, summed in the finalize of the sweep that completes z
      Accum<float> pa[4];
      // B1: y0 = G r (r is the staged centre block of this sweep)
      msweep32(Sv, MP_B1, P.R, nullptr, [&](int row, int a0, int j0, float (&o)[4][4], const float* xc, const float4*, int) {
        for (int r = 0; r < 4; ++r) {
          const size_t idx = (size_t)row * vb + (size_t)(a0 + r) * J + j0;
          const float4 y = make_float4(o[r][0], o[r][1], o[r][2], o[r][3]);
          stv4(P.Y0, idx, y);
          if (m == 1) {
            stv4(P.Z, idx, y);
            const float4 rv = *reinterpret_cast<const float4*>(xc + (a0 + r) * J + j0);
            pa[0].add(rv.x * y.x);
            pa[1].add(rv.y * y.y);
            pa[2].add(rv.z * y.z);
            pa[3].add(rv.w * y.w);
          }
        }
      });
      for (int jp = 1; jp < m && !Sv.fail; ++jp) {
        Sv.barrier();
        const float* yin = (jp == 1) ? P.Y0 : ((jp - 1) % 2 == 1 ? P.Ya : P.Yb);
        float* yout = (jp % 2 == 1) ? P.Ya : P.Yb;
        const float aj = P.alpha[jp];
        const bool lastj = (jp == m - 1);
        msweep32(Sv, MP_B2, yin, lastj ? P.R : nullptr,
                 [&](int row, int a0, int j0, float (&o)[4][4], const float* yc, const float4* rpf, int rst) {
          for (int r = 0; r < 4; ++r) {
            const size_t idx = (size_t)row * vb + (size_t)(a0 + r) * J + j0;
            const float4 y = make_float4(o[r][0], o[r][1], o[r][2], o[r][3]);
            if (!lastj) stv4(yout, idx, y);
            // z so far: y0 (this sweep's staged input row) after the first
            // application of H, else the running sum in Z
            const float4 zp = (jp == 1) ? *reinterpret_cast<const float4*>(yc + (a0 + r) * J + j0) : ldv4(P.Z, idx);
            const float4 z = make_float4(fmaf(aj, y.x, zp.x), fmaf(aj, y.y, zp.y), fmaf(aj, y.z, zp.z),
                                         fmaf(aj, y.w, zp.w));
            stv4(P.Z, idx, z);
            if (lastj) {
              const float4 rv = rpf[r * rst];  // r, staged during the products
              pa[0].add(rv.x * z.x);
              pa[1].add(rv.y * z.y);
              pa[2].add(rv.z * z.z);
              pa[3].add(rv.w * z.w);
            }
          }
        });
      }
      double pv[4];
      widen(pa, pv);
      cta_col_reduce(pv, scratch, colR, ngroups);
      Sv.grid_reduce(colR);
      if (tid < J) rzout[tid] = colR[tid];
      __syncthreads();
    };
    apply_precond(rho);
    // p = z; beta = 0 (with the folded update the first A sweep forms
    // z + 0 p from this copy)
    float* Pc = P.P;   // the current p (the old one while an A sweep folds the update in)
    float* Pn = P.P2;  // where a folding A sweep writes the new p
    {
      const int jg = tid & 15, ag = tid >> 4;
      if (ag < ngroups)
        for (int row = Sv.s; row < Sv.e; ++row)
          for (int r = 0; r < 4; ++r) {
            const size_t idx = (size_t)row * vb + (size_t)(4 * ag + r) * J + 4 * jg;
            stv4(P.P, idx, ldv4(P.Z, idx));
          }
      if (tid < J) betf[tid] = 0.f;
      Sv.barrier();
    }
    // inner iterations
    for (int kit = 1; !Sv.fail; ++kit) {
      const int anyact = __syncthreads_or(tid < J && actv[tid] > 0.0);
      if (!anyact || total_it >= P.maxit) break;
      ++total_it;
      // A: q = S p, pq per column
      Accum<float> pa[4];
      msweep32(Sv, MP_A, Pc, nullptr, [&](int row, int a0, int j0, float (&o)[4][4], const float* pc, const float4*, int) {
        for (int r = 0; r < 4; ++r) {
          const size_t idx = (size_t)row * vb + (size_t)(a0 + r) * J + j0;
          stv4(P.Q, idx, make_float4(o[r][0], o[r][1], o[r][2], o[r][3]));
          const float4 pp = *reinterpret_cast<const float4*>(pc + (a0 + r) * J + j0);
          pa[0].add(pp.x * o[r][0]);
          pa[1].add(pp.y * o[r][1]);
          pa[2].add(pp.z * o[r][2]);
          pa[3].add(pp.w * o[r][3]);
        }
      }, fold ? Fold{P.Z, Pn, betf} : Fold{nullptr, nullptr, nullptr});
      if (fold) {  // the p just formed is the current one
        float* t = Pc;
        Pc = Pn;
        Pn = t;
      }
      double pv[4];
      widen(pa, pv);
      cta_col_reduce(pv, scratch, colR, ngroups);
      Sv.grid_reduce(colR);
      if (tid < J) {
        const double pq = colR[tid];
        if (actv[tid] > 0.0) {
          if (!isfinite(pq)) { actv[tid] = 0.0; outer_act[tid] = -1.0; alp[tid] = 0.0; }
          else if (!(pq > 0.0)) { actv[tid] = 0.0; outer_act[tid] = -2.0; alp[tid] = 0.0; }
          else alp[tid] = rho[tid] / pq;
        } else {
          alp[tid] = 0.0;
        }
        alpf[tid] = (float)alp[tid];
        if (actv[tid] > 0.0) itc[tid] += 1.0;
      }
      __syncthreads();
      // x += alpha p, r -= alpha q, rr per column: the owned rows are one
      // contiguous range of float4s; thread t takes every kMThreads-th (so
      // always column group t % 16) and loads a batch of kVB before storing.
      {
        Accum<float> pa[4];
        const float4 al = *reinterpret_cast<const float4*>(alpf + 4 * (tid & 15));
        const float4* Pp = reinterpret_cast<const float4*>(Pc);
        const float4* Qp = reinterpret_cast<const float4*>(P.Q);
        float4* Xp = reinterpret_cast<float4*>(P.Xin);
        float4* Rp = reinterpret_cast<float4*>(P.R);
        const size_t f1 = (size_t)Sv.e * vb / 4;
        for (size_t f = (size_t)Sv.s * vb / 4 + tid; f < f1; f += (size_t)kVB * kMThreads) {
          float4 pp[kVB], qq[kVB], xx[kVB], rr[kVB];
#pragma unroll
          for (int b = 0; b < kVB; ++b) {
            const size_t g = f + (size_t)b * kMThreads;
            if (g < f1) { pp[b] = Pp[g]; qq[b] = Qp[g]; xx[b] = Xp[g]; rr[b] = Rp[g]; }
          }
#pragma unroll
          for (int b = 0; b < kVB; ++b) {
            const size_t g = f + (size_t)b * kMThreads;
            if (g < f1) {
              Xp[g] = make_float4(fmaf(al.x, pp[b].x, xx[b].x), fmaf(al.y, pp[b].y, xx[b].y),
                                  fmaf(al.z, pp[b].z, xx[b].z), fmaf(al.w, pp[b].w, xx[b].w));
              const float4 rv = make_float4(fmaf(-al.x, qq[b].x, rr[b].x), fmaf(-al.y, qq[b].y, rr[b].y),
                                            fmaf(-al.z, qq[b].z, rr[b].z), fmaf(-al.w, qq[b].w, rr[b].w));
              Rp[g] = rv;
              pa[0].add(rv.x * rv.x);
              pa[1].add(rv.y * rv.y);
              pa[2].add(rv.z * rv.z);
              pa[3].add(rv.w * rv.w);
            }
          }
        }
        double pr[4];
        widen(pa, pr);
        cta_col_reduce(pr, scratch, colR, kMThreads / 16);
        Sv.grid_reduce(colR);
        if (tid < J) {
          rrv[tid] = colR[tid];
          if (actv[tid] > 0.0 && rrv[tid] <= tin[tid]) actv[tid] = 0.0;  // converged column
        }
        __syncthreads();
      }
      const int still = __syncthreads_or(tid < J && actv[tid] > 0.0);
      if (!still) break;
      apply_precond(bet);   // bet temporarily holds the new r.z
      if (tid < J) {
        const double rzn = bet[tid];
        const double b = (actv[tid] > 0.0) ? rzn / rho[tid] : 0.0;
        rho[tid] = rzn;
        bet[tid] = b;
        betf[tid] = (float)b;
      }
      __syncthreads();
      // p = z + beta p, with the access pattern of the x, r update (n > 48;
      // smaller blocks fold it into the next A sweep)
      if (!fold) {
        const float4 be = *reinterpret_cast<const float4*>(betf + 4 * (tid & 15));
        float4* Pp = reinterpret_cast<float4*>(Pc);
        const float4* Zp = reinterpret_cast<const float4*>(P.Z);
        const size_t f1 = (size_t)Sv.e * vb / 4;
        for (size_t f = (size_t)Sv.s * vb / 4 + tid; f < f1; f += (size_t)kVB * kMThreads) {
          float4 pp[kVB], zz[kVB];
#pragma unroll
          for (int b = 0; b < kVB; ++b) {
            const size_t g = f + (size_t)b * kMThreads;
            if (g < f1) { pp[b] = Pp[g]; zz[b] = Zp[g]; }
          }
#pragma unroll
          for (int b = 0; b < kVB; ++b) {
            const size_t g = f + (size_t)b * kMThreads;
            if (g < f1)
              Pp[g] = make_float4(fmaf(be.x, pp[b].x, zz[b].x), fmaf(be.y, pp[b].y, zz[b].y),
                                  fmaf(be.z, pp[b].z, zz[b].z), fmaf(be.w, pp[b].w, zz[b].w));
          }
        }
        Sv.barrier();
      }
    }
    // x64 += ||r64|| * x_in
    {
      const int jg = tid & 15, ag = tid >> 4;
      if (ag < ngroups)
        for (int row = Sv.s; row < Sv.e; ++row)
          for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c) {
              const int j = 4 * jg + c;
              const size_t idx = (size_t)row * vb + (size_t)(4 * ag + r) * J + j;
              if (scl[j] > 0.0) P.X64[idx] = fma(nrv[j], (double)P.Xin[idx], P.X64[idx]);
            }
      Sv.barrier();
    }
  }
  if (Sv.g == 0 && tid < J && tid < P.nrhs) {
    int st = kOK;
    if (Sv.fail) st = kErrTimeout;
    else if (outer_act[tid] == -1.0) st = kErrNonfinite;
    else if (outer_act[tid] == -2.0) st = kErrBreakdown;
    else if (outer_act[tid] > 0.0) st = kErrNoConv;
    else if (!isfinite(nbv[tid])) st = kErrNonfinite;
    P.status[tid] = st;
    P.iters[tid] = (int)itc[tid];
    P.resid[tid] = nbv[tid] > 0.0 ? nrv[tid] / nbv[tid] : 0.0;
    P.outer[tid] = outer;
  }
}

// Layout conversion: caller [N*n][nrhs] (row-major) <-> internal [N][n][kJ].
__global__ void k_mrhs_in(const double* B, double* B64, long long rows, int nrhs) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= rows * kJ) return;
  const long long r = t / kJ;
  const int j = (int)(t % kJ);
  B64[t] = (j < nrhs) ? B[r * nrhs + j] : 0.0;
}
__global__ void k_mrhs_out(const double* X64, double* X, long long rows, int nrhs) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= rows * nrhs) return;
  const long long r = t / nrhs;
  const int j = (int)(t % nrhs);
  X[t] = X64[r * kJ + j];
}

}  // namespace bt

// jobs, plus the staged finalize tiles when the k range is split (n <= 48)
extern "C" int bt_mrhs_smem_bytes(int n) { return kMSmJobs + mrhs_job_bytes(n) + (4 * n <= kMHalf ? 4 * kMHalf * 16 : 0); }

extern "C" cudaError_t bt_launch_mrhs(const bt::MParams* P, const double* B, double* X, int smem, cudaStream_t st) {
  const long long rows = (long long)P->N * P->n;
  const int tb = 256;
  bt::k_mrhs_in<<<(unsigned)((rows * bt::kJ + tb - 1) / tb), tb, 0, st>>>(B, const_cast<double*>(P->B64), rows,
                                                                         P->nrhs);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(bt::bt_mrhs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)P};
  e = cudaLaunchCooperativeKernel((const void*)bt::bt_mrhs_kernel, dim3(P->G), dim3(bt::kMThreads), args, smem, st);
  if (e != cudaSuccess) return e;
  bt::k_mrhs_out<<<(unsigned)((rows * P->nrhs + tb - 1) / tb), tb, 0, st>>>(P->X64, X, rows, P->nrhs);
  return cudaGetLastError();
}

extern "C" cudaError_t bt_mrhs_occupancy(int smem, int* blocks) {
  cudaError_t e = cudaFuncSetAttribute(bt::bt_mrhs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, bt::bt_mrhs_kernel, bt::kMThreads, smem);
}

// Host launcher: fills the kernel parameters from plain pointers (the
// workspace vector list is B64, X64, R64, Xin, R, P, Q, Y0, Ya, Yb, Z, red,
// ctl, int results [iters | status | outer], double results [resid], P2).
extern "C" cudaError_t bt_mrhs_solve_launch(int N, int n, int m, const double* alpha, const float* const* blk32,
                                            const double* D64, const double* O64, int bs32, int bs64,
                                            void* const* vec, double tol, double tol_inner, int maxit,
                                            int max_outer, long long budget, int G, int nrhs, const double* B,
                                            double* X, int smem, cudaStream_t st) {
  bt::MParams P{};
  P.D32 = blk32[0]; P.O32 = blk32[1]; P.Dinv32 = blk32[2]; P.E32 = blk32[3];
  P.Hd32 = blk32[4]; P.Hu32 = blk32[5]; P.Hl32 = blk32[6];
  P.D64 = D64;
  P.O64 = O64;
  P.N = N; P.n = n; P.bs32 = bs32; P.bs64 = bs64; P.m = m;
  for (int j = 0; j < bt::kMaxM; ++j) P.alpha[j] = j < m ? (float)alpha[j] : 0.0f;
  P.B64 = static_cast<const double*>(vec[0]);
  P.X64 = static_cast<double*>(vec[1]);
  P.R64 = static_cast<double*>(vec[2]);
  P.Xin = static_cast<float*>(vec[3]);
  P.R = static_cast<float*>(vec[4]);
  P.P = static_cast<float*>(vec[5]);
  P.Q = static_cast<float*>(vec[6]);
  P.Y0 = static_cast<float*>(vec[7]);
  P.Ya = static_cast<float*>(vec[8]);
  P.Yb = static_cast<float*>(vec[9]);
  P.Z = static_cast<float*>(vec[10]);
  P.P2 = static_cast<float*>(vec[15]);
  P.red = static_cast<double*>(vec[11]);
  int* ctl = static_cast<int*>(vec[12]);
  P.abort_flag = ctl + 1;
  P.bar = reinterpret_cast<unsigned*>(ctl + 2);
  int* ri = static_cast<int*>(vec[13]);
  P.iters = ri;
  P.status = ri + bt::kJ;
  P.outer = ri + 2 * bt::kJ;
  P.resid = static_cast<double*>(vec[14]);
  P.tol = tol;
  P.tol_inner = tol_inner;
  P.maxit = maxit;
  P.max_outer = max_outer;
  P.budget = budget;
  P.G = G;
  P.nrhs = nrhs;
  return bt_launch_mrhs(&P, B, X, smem, st);
}
