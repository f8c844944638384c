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
#include <algorithm>
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
  // Tensor-core engine: per block row, the block Q of each product out = Q x
  // as a K-major core-matrix image (see k_mrhs_image), n*n floats per row:
  // role 0 (block (c, c)): D, D^-1, Hd; role 1 (block (c+k, c)): O^T, -E^T, Hl;
  // role 2 (block (c-k, c), stored at index c-k): O, -E, Hu.
  const float *img_d, *img_dinv, *img_hd, *img_ot, *img_et, *img_hl, *img_o, *img_e, *img_hu;
  int N, n, bs32, bs64, m;
  float alpha[kMaxM];
  // float64 vectors [N][n][J]
  const double* B64;
  double* X64;
  double* R64;
  // float32 vectors [N][n][J]
  float *Xin, *R, *P, *Q, *Y0, *Ya, *Yb, *Z;
  float* P2;            // second p buffer: the A sweep writes the new p there (n <= 48)
  float* R2;            // second r buffer: the tensor-core B1 sweep writes the new r there (m >= 2)
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
  double* colred;   // smem scratch for the cross-CTA column sums ([kMThreads / kJ][kJ])
  // tensor-core engine: TMEM base address, and the counts behind the mbarrier
  // phases (identical in every thread): columns whose data was waited for /
  // issued, MMA commits waited for / issued
  unsigned tmem;
  int gcol, iss, mma_done, mma_iss;

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
      for (int b0 = g0; b0 < g1; b0 += 16) {  // 16 loads in flight, then the adds in slot order
        double v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) v[u] = (b0 + u < g1) ? __ldcg(src + (size_t)(b0 + u) * kJ) : 0.0;
#pragma unroll
        for (int u = 0; u < 16; ++u)
          if (b0 + u < g1) t += v[u];
      }
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

  // Grid barrier alone (no values): the arrival count of grid_reduce.
  // Bounded.
  __device__ void barrier() {
    if (fail) return;
    __syncthreads();
    int* flag = reinterpret_cast<int*>(sm);
    ++bar_count;  // the reductions' slot parity counts these barriers too
    if (threadIdx.x == 0) {
      __threadfence();  // publishes the CTA's global writes before the arrival
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
    if (flag[0]) fail = true;
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
  int sq;  // tensor-core B1 fold: sum (new r)^2 over the owned rows, this thread's part to the column scratch
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

// ------------------------------------------------------------ tensor cores
// The tensor-core engine (row of the many-RHS path where the work is a dense
// contraction): every product out = Q x of a sweep is an n x n by n x 64
// contraction, computed transposed, out^T = x^T Q^T, by tcgen05.mma kind::tf32
// with N = n and K = 8 per instruction, accumulating in tensor memory (TMEM).
// Both operands are K-major
// SWIZZLE_NONE core-matrix images in shared memory: 8 rows x 16 bytes per core
// matrix, element (row a, k) of an operand at
//     ((a / 8) * (n / 4) + k / 4) * 32 + (a % 8) * 4 + k % 4     (floats),
// so the K-direction core stride (LBO) is 128 bytes and the 8-row stride
// (SBO) 32 n bytes.  Float32 accuracy from TF32 units: each operand is split
// x = hi + lo with hi = tf32(x) and lo = tf32(x - hi) (rounded: the tensor
// cores read the top 19 bits of each operand and drop the rest).  The A
// operand stacks the two parts of the vector row, [x_hi^T; x_lo^T], into
// M = 128 rows, so that per K step two MMAs (with Q_hi and Q_lo) form all four
// partial products: TMEM lane j < 64 accumulates x_hi^T Q^T + x_hi^T Q_lo^T
// for right-hand side j, lane 64 + j the x_lo terms; the finalize adds the two
// (float32 accumulation throughout).  Row i of the M = 128 accumulator is
// TMEM lane i, column r of out^T TMEM column r.
constexpr int kTcMaxN = 48;
constexpr unsigned kTmemCols = 512;

__device__ __forceinline__ uint64_t tc_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor: D float32, A and B tf32, both K-major, M = 128, N = n
__device__ __forceinline__ unsigned tc_idesc(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(n >> 3) << 17) | (8u << 24);
}
// thread that issues the MMAs and the bulk copies: lane 0 of the last warp,
// which holds no finalize tile and reads no TMEM
constexpr int kTcIssuer = kMThreads - 32;
__device__ __forceinline__ void tc_mma(unsigned d, uint64_t a, uint64_t b, unsigned id, unsigned acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}
// the mbarrier completes once every MMA this thread issued before it has finished
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// 8 consecutive TMEM columns of the warp's 32 lanes (lane = thread)
__device__ __forceinline__ void tc_ld8(unsigned ta, float (&v)[8]) {
  unsigned r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(ta)
               : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tc_alloc(unsigned* slot) {  // one warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(kTmemCols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(unsigned taddr) {  // one warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTmemCols) : "memory");
}
// x rounded to TF32 (11 significant bits, ties away from zero) on its bit pattern
__device__ __forceinline__ float tf32_round(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
}
__device__ __forceinline__ void split4(const float4 v, float4& h, float4& l) {
  h = make_float4(tf32_round(v.x), tf32_round(v.y), tf32_round(v.z), tf32_round(v.w));
  l = make_float4(tf32_round(v.x - h.x), tf32_round(v.y - h.y), tf32_round(v.z - h.z), tf32_round(v.w - h.w));
}
__device__ __forceinline__ float comp(const float4& v, int i) { return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w)); }

// Shared memory of the tensor-core sweeps (floats, from kTcBase: the column
// sums' scratch and the SIMT exchange tiles are idle during a sweep):
//   bimg  [2][3][2][n n]  per column buffer, blocks of rows c - k, c, c + k: [hi | lo] B images (one
//                         bulk copy of the block's [hi | lo] image)
//   aimg  [2][64 n]       [hi; lo] A image of the column's vector row
//   ring  [3][n 64]       raw vector rows (columns c .. c + 2)
//   stage [2][n 64]       the finished row, [n][64]: x_hi and x_lo partial sums
//   fbuf  [2][n 64]       the finished row's input and `pre` tiles ([n][64],
//                         each finalize thread copies and reads its own tile)
constexpr int kTcBase = kMSmScratch;
__host__ __device__ constexpr int mrhs_tc_floats(int n) { return 12 * n * n + 9 * n * kJ; }
constexpr int kTcBarOff = 64;  // bytes: full[2], mma, TMEM slot (in the flag words)

// One sweep (A, B1 or B2) on the tensor cores, in column form: column c's
// vector row x_c multiplies the three blocks of block column c, accumulating
// into rows c - k, c, c + k (k = 2 for H, else 1).  Per block and K step one
// MMA with A = [x_hi; x_lo] (M = 128) and B = [Q_hi | Q_lo] (N = 2n) forms the
// four partial products of x^T Q^T into the row's TMEM accumulator (2k + 1 of
// them, 2n columns each).  Step c of the loop:
//   the finalize threads start copying the input (and `pre`) tiles of row
//   t = c - 1 - k; wait for column c's data (issued two steps earlier); split
//   it into TF32 parts; read row t (complete since column c - 1's MMAs, the
//   last with a product into it, were waited for) from TMEM; issue the MMAs
//   of column c (whose new row c + k reuses row t's slot); finalize row t
//   from shared memory while they run; wait for them and issue the bulk
//   copies of column c + 2 into the buffers they released.
// A CTA processes the columns s - k .. e + k - 1 of its rows [s, e); a halo
// column contributes to the owned rows only.  One thread (kTcIssuer) issues
// the bulk copies and the MMAs; warps 0-7 read TMEM; the finalize tiles run on
// threads < 4n.
// `fd` (A sweep): the p update folded in -- the split forms p = z + beta p_old
// from the copied p_old row and the z row (staged by cp.async into the `pre`
// tile buffer, free in this sweep, one column ahead by the threads with no
// finalize tile), writes p of the owned rows to fd.pout and feeds the MMAs
// with it; the finalize reads its p tile from fd.pout.  Halo columns form
// their p the same way (p_old and z of the neighbours are not rewritten
// during the sweep).  `fd` (B1 sweep): the r update r = r_old - alpha q folded
// in the same way (fd.z = q, fd.beta = alpha); with fd.sq each thread sums the
// new r^2 of its column (tid % 64) over the owned rows and leaves the sum in
// the column scratch, [tid / 64][tid % 64], when the sweep ends.
template <typename Fin>
__device__ void msweep_tc(MSolver& Sv, int phase, const float* v_in, const float* pre, Fin fin, const Fold& fd) {
  const MParams& P = Sv.P;
  const int n = Sv.n, N = Sv.N, s = Sv.s, e = Sv.e;
  __syncthreads();
  if (e <= s || Sv.fail) return;
  const int tid = threadIdx.x;
  const int k = (phase == MP_B2) ? 2 : 1;
  const int S = 2 * k + 1;
  const int slot_cols = (2 * n + 31) / 32 * 32;
  const int bb = n * n, vb = n * kJ, nk4 = n / 4;
  const int c_lo = max(0, s - k), c_hi = min(N, e + k);
  const float* img0 = phase == MP_A ? P.img_d : (phase == MP_B1 ? P.img_dinv : P.img_hd);
  const float* img1 = phase == MP_A ? P.img_ot : (phase == MP_B1 ? P.img_et : P.img_hl);
  const float* img2 = phase == MP_A ? P.img_o : (phase == MP_B1 ? P.img_e : P.img_hu);
  float* bimg = reinterpret_cast<float*>(Sv.sm + kTcBase);
  float* aimg = bimg + 12 * bb;
  float* ring = aimg + 2 * vb;
  float* stage = ring + 3 * vb;
  float* xbuf = stage + 2 * vb;
  float* pbuf = xbuf + vb;
  uint64_t* full = reinterpret_cast<uint64_t*>(Sv.sm + kTcBarOff);
  uint64_t* mbar = full + 2;
  // images in the order role 2, 0, 1 (rows c - k, c, c + k): the blocks of
  // rows c - k and c are adjacent, one B operand of N = 4n
  const auto bptr = [&](int buf, int role) { return bimg + (size_t)(buf * 3 + (role + 1) % 3) * 2 * bb; };
  // TMEM slot of row t: t m mod S with m k = 1 (mod S), so that rows c - k,
  // c, c + k sit in consecutive slots (mod S)
  const int mslot = (k == 1) ? 1 : 3;
  const auto tslot = [&](int t) { return (t * mslot) % S; };
  // rows c - k and c share one MMA of N = 4n when their slots are adjacent in
  // TMEM (not wrapped) and a slot is exactly the 2n columns of a row
  const bool can_merge = slot_cols == 2 * n;
  const auto slot = [&](int r) { return ring + (size_t)(r % 3) * vb; };
  // role 0: row c (block (c, c)); 1: row c + k; 2: row c - k
  const auto target = [&](int c, int role) { return role == 0 ? c : (role == 1 ? c + k : c - k); };
  const auto role_ok = [&](int c, int role) {
    const int t = target(c, role);
    return t >= s && t < e && t < N;
  };
  const auto issue = [&](int c, int buf) {  // kTcIssuer
    unsigned bytes = (unsigned)vb * 4u;
    for (int r = 0; r < 3; ++r)
      if (role_ok(c, r)) bytes += (unsigned)bb * 8u;
    mbar_arrive_expect_tx(full + buf, bytes);
    for (int r = 0; r < 3; ++r) {
      if (!role_ok(c, r)) continue;
      const size_t blk = r == 2 ? (size_t)(c - k) : (size_t)c;
      const float* src = (r == 0 ? img0 : (r == 1 ? img1 : img2)) + blk * 2 * bb;
      bulk_g2s(bptr(buf, r), src, (unsigned)bb * 8u, full + buf);  // [hi | lo]
    }
    bulk_g2s(slot(c), v_in + (size_t)c * vb, (unsigned)vb * 4u, full + buf);
  };
  if (tid == kTcIssuer) {
    fence_proxy_async_smem();
    if (c_lo < c_hi) issue(c_lo, Sv.gcol & 1);
    if (c_lo + 1 < c_hi) issue(c_lo + 1, (Sv.gcol + 1) & 1);
  }
  Sv.iss = Sv.gcol + min(2, c_hi - c_lo);
  const int a0 = 4 * (tid >> 4), j0 = 4 * (tid & 15);  // finalize tile of threads < 4n
  const bool fold = fd.z != nullptr && (phase == MP_A || phase == MP_B1);
  const float* fin_src = fold ? fd.pout : v_in;  // the finalize's input tile
  // threads with neither a finalize tile nor the copy / MMA issue
  const int sp0 = (4 * n + 31) / 32 * 32, spn = kTcIssuer - sp0;
  Accum<float> sqa;  // fd.sq: this thread's sum of the new r^2
  // z row cc into pbuf (threads sp0 .. kTcIssuer - 1)
  const auto stage_z = [&](int cc) {
    if (tid >= sp0 && tid < kTcIssuer) {
      for (int f = tid - sp0; f < vb / 4; f += spn) cp16(pbuf + 4 * f, fd.z + (size_t)cc * vb + 4 * f);
      cp_commit();
    }
  };
  if (fold && c_lo < c_hi) stage_z(c_lo);
  bool bad = false;
  for (int c = c_lo; c <= e + k; ++c) {  // step e + k finishes row e - 1
    const bool proc = c < c_hi;
    const int buf = Sv.gcol & 1;  // buffers of column c (global column index gcol)
    const int t = c - 1 - k;      // the row this step finishes
    const bool fin_t = t >= s && t < e;
    if (fin_t && tid < 4 * n) {  // this thread's input (and pre) tile of row t
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const size_t g = (size_t)t * vb + (size_t)(a0 + r) * kJ + j0;
        cp16(xbuf + (a0 + r) * kJ + j0, fin_src + g);
        if (pre) cp16(pbuf + (a0 + r) * kJ + j0, pre + g);
      }
      cp_commit();
    }
    if (proc) {
      if (fold && tid >= sp0 && tid < kTcIssuer) cp_wait<0>();  // this thread's part of z row c
      const bool ok = mbar_wait(full + buf, (unsigned)((Sv.gcol >> 1) & 1), Sv.deadline);
      if (__syncthreads_or(!ok)) {
        bad = true;
        break;
      }
      // split the vector row (transposed into the A image: one right-hand side
      // j and four k per task); the blocks arrive split ([hi | lo] images)
      const float* xr = slot(c);
      const bool own_c = c >= s && c < e;
      for (int q = tid; q < 16 * n; q += kMThreads) {
        const int j = q & 63, k4 = q >> 6;
        float4 x = make_float4(xr[(4 * k4) * kJ + j], xr[(4 * k4 + 1) * kJ + j], xr[(4 * k4 + 2) * kJ + j],
                               xr[(4 * k4 + 3) * kJ + j]);
        if (fold) {
          const float bj = fd.beta[j];
          const float* zr = pbuf + (4 * k4) * kJ + j;
          if (phase == MP_A)  // p = z + beta_j p_old
            x = make_float4(fmaf(bj, x.x, zr[0]), fmaf(bj, x.y, zr[kJ]), fmaf(bj, x.z, zr[2 * kJ]),
                            fmaf(bj, x.w, zr[3 * kJ]));
          else  // r = r_old - alpha_j q
            x = make_float4(fmaf(-bj, zr[0], x.x), fmaf(-bj, zr[kJ], x.y), fmaf(-bj, zr[2 * kJ], x.z),
                            fmaf(-bj, zr[3 * kJ], x.w));
          if (own_c) {
            float* po = fd.pout + (size_t)c * vb + (size_t)(4 * k4) * kJ + j;
            po[0] = x.x;
            po[kJ] = x.y;
            po[2 * kJ] = x.z;
            po[3 * kJ] = x.w;
            if (fd.sq) {
              sqa.add(x.x * x.x);
              sqa.add(x.y * x.y);
              sqa.add(x.z * x.z);
              sqa.add(x.w * x.w);
            }
          }
        }
        float4 h, l;
        split4(x, h, l);
        const int off = ((j >> 3) * nk4 + k4) * 32 + (j & 7) * 4;
        *reinterpret_cast<float4*>(aimg + off) = h;
        *reinterpret_cast<float4*>(aimg + vb + off) = l;
      }
    } else if (fin_t) {
      __syncthreads();  // the previous finalize has read the stage
    }
    if (fin_t) {  // read row t from TMEM
      tc_fence_after();
      const int warp = tid >> 5, lane = tid & 31, q = warp & 3;
      if (warp < 8) {  // lanes 0-63: x_hi terms of column j = lane + 32 q; 64-127: x_lo terms
        const unsigned base = Sv.tmem + (unsigned)(tslot(t) * slot_cols) + ((unsigned)(32 * q) << 16);
        float* st = stage + (q >> 1) * vb + 32 * (q & 1) + lane;
        for (int ch = warp >> 2; ch < n / 8; ch += 2) {
          float v[8], w[8];
          tc_ld8(base + 8u * (unsigned)ch, v);                // x Q_hi^T
          tc_ld8(base + (unsigned)n + 8u * (unsigned)ch, w);  // x Q_lo^T
#pragma unroll
          for (int i = 0; i < 8; ++i) st[(8 * ch + i) * kJ] = v[i] + w[i];
        }
      }
    }
    if (proc || fin_t) {
      fence_proxy_async_smem();
      tc_fence_before();
      __syncthreads();
    }
    // the z row of the next column into pbuf (the split of this one has read it)
    if (fold && proc && c + 1 < c_hi) stage_z(c + 1);
    if (proc) {
      if (tid == kTcIssuer) {
        tc_fence_after();
        const unsigned id = tc_idesc(2 * n);
        const unsigned sbo = 32u * (unsigned)n;
        // descriptors of K step 0; step ks starts 256 ks bytes later (16 ks in
        // the address field)
        const uint64_t da = tc_desc(smem_u32(aimg), 128, sbo);  // [x_hi; x_lo]
        // rows c - k and c both accumulate (row c - k had its first product
        // from column c - 2k, row c from column c - k, which exists when row
        // c - k does)
        const bool merge = can_merge && role_ok(c, 2) && role_ok(c, 0) && tslot(c - k) != S - 1;
        if (merge) {
          const unsigned id2 = tc_idesc(4 * n);
          const unsigned d = Sv.tmem + (unsigned)(tslot(c - k) * slot_cols);
          const uint64_t db = tc_desc(smem_u32(bptr(buf, 2)), 128, sbo);  // [Q2_hi | Q2_lo | Q0_hi | Q0_lo]
          for (int ks = 0; ks < n / 8; ++ks) {
            const uint64_t o = 16ull * (unsigned)ks;
            tc_mma(d, da + o, db + o, id2, 1u);
          }
        }
        for (int r = 0; r < 3; ++r) {
          if (!role_ok(c, r) || (merge && r != 1)) continue;
          const int tr = target(c, r);
          // the first product into a row: role 1, or role 0 when column c - k does not exist
          const bool first = (r == 1) || (r == 0 && c - k < 0);
          const unsigned d = Sv.tmem + (unsigned)(tslot(tr) * slot_cols);
          const uint64_t db = tc_desc(smem_u32(bptr(buf, r)), 128, sbo);  // [Q_hi | Q_lo]
          for (int ks = 0; ks < n / 8; ++ks) {
            const uint64_t o = 16ull * (unsigned)ks;
            tc_mma(d, da + o, db + o, id, (first && ks == 0) ? 0u : 1u);
          }
        }
        tc_commit(mbar);
      }
      ++Sv.mma_iss;
    }
    if (fin_t && tid < 4 * n) {
      cp_wait<0>();  // this thread's own tiles
      float out[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float4 w = *reinterpret_cast<const float4*>(stage + (a0 + r) * kJ + j0);
        const float4 x = *reinterpret_cast<const float4*>(stage + vb + (a0 + r) * kJ + j0);
        out[r][0] = w.x + x.x; out[r][1] = w.y + x.y; out[r][2] = w.z + x.z; out[r][3] = w.w + x.w;
      }
      fin(t, a0, j0, out, xbuf, pre ? reinterpret_cast<const float4*>(pbuf + a0 * kJ + j0) : nullptr, kJ / 4);
    }
    if (proc) {
      const bool ok = mbar_wait(mbar, (unsigned)(Sv.mma_done & 1), Sv.deadline);
      if (__syncthreads_or(!ok)) {
        bad = true;
        break;
      }
      ++Sv.mma_done;
      ++Sv.gcol;
      if (c + 2 < c_hi) {  // column c + 2 into the buffers column c released
        if (tid == kTcIssuer) {
          fence_proxy_async_smem();
          issue(c + 2, buf);
        }
        ++Sv.iss;
      }
    }
  }
  if (bad) {
    // let every copy and MMA this CTA started finish (bounded) before the
    // kernel goes on to release TMEM and exit
    const long long lim = clock64() + (1ll << 31);
    cp_wait<0>();
    for (int gc = Sv.gcol; gc < Sv.iss; ++gc) mbar_wait(full + (gc & 1), (unsigned)((gc >> 1) & 1), lim);
    for (int m = Sv.mma_done; m < Sv.mma_iss; ++m) mbar_wait(mbar, (unsigned)(m & 1), lim);
    Sv.gcol = Sv.iss;
    Sv.mma_done = Sv.mma_iss;
    Sv.fail = true;
    if (tid == 0) atomicExch(P.abort_flag, 1);
  }
  __syncthreads();
  // the column scratch overlaps the sweep's buffers, idle now
  if (fold && fd.sq) Sv.colred[(tid / kJ) * kJ + tid % kJ] = sqa.value();
}

template <bool TC, typename Fin>
__device__ __forceinline__ void msweep(MSolver& Sv, int phase, const float* v_in, const float* pre, Fin fin,
                                       const Fold& fd = Fold{nullptr, nullptr, nullptr}) {
  if constexpr (TC) msweep_tc(Sv, phase, v_in, pre, fin, fd);
  else msweep32(Sv, phase, v_in, pre, fin, fd);
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
// TC: block products on the tensor cores (msweep_tc), else float32 SIMT tiles.
template <bool TC>
__global__ void __launch_bounds__(kMThreads, 1) bt_mrhs_kernel(const __grid_constant__ MParams P) {
  extern __shared__ __align__(128) char smem[];
  MSolver Sv(P, smem);
  Sv.tmem = 0;
  Sv.gcol = Sv.iss = Sv.mma_done = Sv.mma_iss = 0;
  if constexpr (TC) {
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kTcBarOff);
    unsigned* tslot = reinterpret_cast<unsigned*>(smem + kTcBarOff + 24);
    if (threadIdx.x == 0) {
      for (int b = 0; b < 3; ++b) mbar_init(bars + b, 1);
      fence_mbar_init();
    }
    if (threadIdx.x < 32) tc_alloc(tslot);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    Sv.tmem = *tslot;
  }
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
  float* alpq = reinterpret_cast<float*>(col + 2 * kJ);  // float alpha of the previous iteration
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
  Sv.colred = scratch;
  const int n = P.n;
  const int tid = threadIdx.x;
  const int ngroups = n / 4;
  const size_t vb = (size_t)n * kJ;
  const int J = kJ;
  const int m = P.m;
  const bool fold = TC || 4 * n <= kMHalf;  // p update folded into the A sweep (SIMT: the k-split layout)
  const bool foldr = TC && m >= 2;  // r update folded into the B1 sweep (tensor cores, with H sweeps)

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
    float* Rc = P.R;   // the current r
    float* Rn = P.R2;  // where a B1 sweep with the r update folded in writes the new r
    // z0 = M^-1 r0 ; rho = r.z.  fr (foldr): the B1 sweep first forms
    // r = r_old - alpha q (r.r per column reduced after it, the barrier before
    // the H sweeps); returns true when no column remains active (the H sweeps
    // are then skipped).
    auto apply_precond = [&](double* rzout, bool fr) -> bool {
      // r.z per column, summed in the finalize of the sweep that completes z
      Accum<float> pa[4];
      // B1: y0 = G r (r is the staged centre block of this sweep)
      msweep<TC>(Sv, MP_B1, Rc, nullptr, [&](int row, int a0, int j0, float (&o)[4][4], const float* xc, const float4*, int) {
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
      }, fr ? Fold{P.Q, Rn, alpf, 1} : Fold{nullptr, nullptr, nullptr, 0});
      if (fr) {
        float* t = Rc;  // the r just formed is the current one
        Rc = Rn;
        Rn = t;
        // r.r per column (the sweep left each thread's part in the scratch),
        // then over the grid
        __syncthreads();
        if (tid < kJ) {
          double sum = 0.0;
          for (int a = 0; a < kMThreads / kJ; ++a) sum += scratch[a * kJ + tid];
          colR[tid] = sum;
        }
        __syncthreads();
        Sv.grid_reduce(colR);
        if (tid < J) {
          rrv[tid] = colR[tid];
          if (actv[tid] > 0.0 && rrv[tid] <= tin[tid]) actv[tid] = 0.0;  // converged column
        }
        __syncthreads();
        if (!__syncthreads_or(tid < J && actv[tid] > 0.0)) return true;
      }
      for (int jp = 1; jp < m && !Sv.fail; ++jp) {
        if (!(fr && jp == 1)) Sv.barrier();  // (fr: the r.r reduction was the barrier)
        const float* yin = (jp == 1) ? P.Y0 : ((jp - 1) % 2 == 1 ? P.Ya : P.Yb);
        float* yout = (jp % 2 == 1) ? P.Ya : P.Yb;
        const float aj = P.alpha[jp];
        const bool lastj = (jp == m - 1);
        msweep<TC>(Sv, MP_B2, yin, lastj ? Rc : nullptr,
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
      return false;
    };
    apply_precond(rho, false);
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
    // x += alpha p over the owned rows (the current p and alpha: Pc, alpf),
    // or x += alpha' p' + alpha p (two): p' = Pn with alpha' = alpq first
    bool x_pending = false;
    auto x_update = [&](bool two) {
      const float4 al = *reinterpret_cast<const float4*>(alpf + 4 * (tid & 15));
      const float4 a2 = *reinterpret_cast<const float4*>(alpq + 4 * (tid & 15));
      const float4* Pp = reinterpret_cast<const float4*>(Pc);
      const float4* P2p = reinterpret_cast<const float4*>(Pn);
      float4* Xp = reinterpret_cast<float4*>(P.Xin);
      const size_t f1 = (size_t)Sv.e * vb / 4;
      // loads of a batch of kVB before its stores: one latency per batch
      for (size_t f = (size_t)Sv.s * vb / 4 + tid; f < f1; f += (size_t)kVB * kMThreads) {
        float4 xx[kVB], pp[kVB], qq[kVB];
#pragma unroll
        for (int b = 0; b < kVB; ++b) {
          const size_t g = min(f + (size_t)b * kMThreads, f1 - 1);  // clamped: loads stay in range
          xx[b] = Xp[g];
          pp[b] = Pp[g];
          qq[b] = two ? P2p[g] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int b = 0; b < kVB; ++b) {
          const size_t g = f + (size_t)b * kMThreads;
          float4 x = xx[b];
          if (two)
            x = make_float4(fmaf(a2.x, qq[b].x, x.x), fmaf(a2.y, qq[b].y, x.y), fmaf(a2.z, qq[b].z, x.z),
                            fmaf(a2.w, qq[b].w, x.w));
          if (g < f1)
            Xp[g] = make_float4(fmaf(al.x, pp[b].x, x.x), fmaf(al.y, pp[b].y, x.y), fmaf(al.z, pp[b].z, x.z),
                                fmaf(al.w, pp[b].w, x.w));
        }
      }
    };
    // inner iterations
    for (int kit = 1; !Sv.fail; ++kit) {
      const int anyact = __syncthreads_or(tid < J && actv[tid] > 0.0);
      if (!anyact || total_it >= P.maxit) break;
      ++total_it;
      // A: q = S p, pq per column
      Accum<float> pa[4];
      msweep<TC>(Sv, MP_A, Pc, nullptr, [&](int row, int a0, int j0, float (&o)[4][4], const float* pc, const float4*, int) {
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
        double a = 0.0;
        if (actv[tid] > 0.0) {
          if (!isfinite(pq)) { actv[tid] = 0.0; outer_act[tid] = -1.0; }
          else if (!(pq > 0.0)) { actv[tid] = 0.0; outer_act[tid] = -2.0; }
          else a = rho[tid] / pq;
        }
        alpq[tid] = alpf[tid];  // the previous iteration's alpha (paired x updates)
        alpf[tid] = (float)a;
        if (actv[tid] > 0.0) itc[tid] += 1.0;
      }
      __syncthreads();
      if (foldr) {
        // x += alpha p over the owned rows (no other CTA reads them: no
        // barrier); r and r.r are formed in the B1 sweep.  Two iterations per
        // pass: an odd one leaves alpha_k p_k pending (p_k stays in Pc, then
        // in Pn until the A sweep after next), an even one adds
        // alpha_{k-1} p_{k-1} + alpha_k p_k (the same fma sequence)
        if (kit & 1) x_pending = true;
        else {
          x_update(true);
          x_pending = false;
        }
      } else {
        // x += alpha p, r -= alpha q, rr per column: the owned rows are one
        // contiguous range of float4s; thread t takes every kMThreads-th (so
        // always column group t % 16) and loads a batch of kVB before storing.
        {
          Accum<float> pa[4];
          const float4 al = *reinterpret_cast<const float4*>(alpf + 4 * (tid & 15));
          const float4* Pp = reinterpret_cast<const float4*>(Pc);
          const float4* Qp = reinterpret_cast<const float4*>(P.Q);
          float4* Xp = reinterpret_cast<float4*>(P.Xin);
          float4* Rp = reinterpret_cast<float4*>(Rc);
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
      }
      if (apply_precond(bet, foldr)) break;  // bet temporarily holds the new r.z
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
    if (x_pending) {  // the last odd iteration's alpha p
      x_update(false);
      __syncthreads();  // x_in is read below with another thread mapping
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
  if constexpr (TC) {  // every MMA was waited for (or drained after a timeout)
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
      tc_fence_after();
      tc_dealloc(Sv.tmem);
    }
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

// Q_i as the K-major core-matrix image of the tensor-core engine: element
// (a, b) of Q_i at ((a / 8) * (n / 4) + b / 4) * 32 + (a % 8) * 4 + b % 4,
// Q_i = sign * M_i (trans = 0) or sign * M_i^T (trans = 1), M_i read from the
// library's column-major float32 slot (M_i(a, b) at b * n + a).
__global__ void k_mrhs_image(const float* src, int bs32, float* dst, int N, int n, int trans, float sign) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long bb = (long long)n * n;
  if (t >= (long long)N * bb) return;
  const long long i = t / bb;
  const int w = (int)(t - i * bb);
  const int a = w / n, b = w - (w / n) * n;
  const float v = sign * (trans ? src[i * bs32 + (long long)a * n + b] : src[i * bs32 + (long long)b * n + a]);
  // [hi | lo] TF32 parts of block row i, 2 n^2 floats: the B operand of the
  // sweep's MMAs as it lands in shared memory
  const float h = tf32_round(v);
  const long long o = i * 2 * bb + ((a >> 3) * (n >> 2) + (b >> 2)) * 32 + (a & 7) * 4 + (b & 3);
  dst[o] = h;
  dst[o + bb] = tf32_round(v - h);
}

}  // namespace bt

// Shared memory of the many-RHS kernel: the common prefix, then the jobs (plus
// the staged finalize tiles when the k range is split, n <= 48) for the SIMT
// engine, or the tensor-core sweep buffers (which also hold the float64
// residual sweep's job).
extern "C" int bt_mrhs_smem_bytes(int n, int tc) {
  if (tc) return std::max(kTcBase + bt::mrhs_tc_floats(n) * 4, kMSmJobs + mrhs_job_bytes(n));
  return kMSmJobs + mrhs_job_bytes(n) + (4 * n <= kMHalf ? 4 * kMHalf * 16 : 0);
}

extern "C" int bt_mrhs_tc_supported(int n) { return n % 8 == 0 && n >= 8 && n <= bt::kTcMaxN; }

static const void* mrhs_kernel(int tc) {
  return tc ? (const void*)bt::bt_mrhs_kernel<true> : (const void*)bt::bt_mrhs_kernel<false>;
}

extern "C" cudaError_t bt_launch_mrhs(const bt::MParams* P, const double* B, double* X, int smem, int tc,
                                      cudaStream_t st) {
  const long long rows = (long long)P->N * P->n;
  const int tb = 256;
  bt::k_mrhs_in<<<(unsigned)((rows * bt::kJ + tb - 1) / tb), tb, 0, st>>>(B, const_cast<double*>(P->B64), rows,
                                                                         P->nrhs);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const void* kern = mrhs_kernel(tc);
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)P};
  e = cudaLaunchCooperativeKernel(kern, dim3(P->G), dim3(bt::kMThreads), args, smem, st);
  if (e != cudaSuccess) return e;
  bt::k_mrhs_out<<<(unsigned)((rows * P->nrhs + tb - 1) / tb), tb, 0, st>>>(P->X64, X, rows, P->nrhs);
  return cudaGetLastError();
}

extern "C" cudaError_t bt_mrhs_occupancy(int smem, int tc, int* blocks) {
  const void* kern = mrhs_kernel(tc);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern, bt::kMThreads, smem);
}

// The nine block images of the tensor-core engine from the float32 slots
// (img: D, D^-1, Hd, O^T, -E^T, Hl, O, -E, Hu; H images only for m >= 2).
extern "C" cudaError_t bt_mrhs_images(int N, int n, int m, const float* const* blk32, int bs32, float* const* img,
                                      cudaStream_t st) {
  // blk32: D, O, D^-1, E, Hd, Hu, Hl
  const float* src[9] = {blk32[0], blk32[2], blk32[4], blk32[1], blk32[3], blk32[6], blk32[1], blk32[3], blk32[5]};
  const int trans[9] = {0, 0, 0, 1, 1, 0, 0, 0, 0};
  const float sign[9] = {1.f, 1.f, 1.f, 1.f, -1.f, 1.f, 1.f, -1.f, 1.f};
  const long long tot = (long long)N * n * n;
  const int tb = 256;
  for (int i = 0; i < 9; ++i) {
    if ((i == 2 || i == 5 || i == 8) && m < 2) continue;
    bt::k_mrhs_image<<<(unsigned)((tot + tb - 1) / tb), tb, 0, st>>>(src[i], bs32, img[i], N, n, trans[i], sign[i]);
  }
  return cudaGetLastError();
}

// Host launcher: fills the kernel parameters from plain pointers (the
// workspace vector list is B64, X64, R64, Xin, R, P, Q, Y0, Ya, Yb, Z, red,
// ctl, int results [iters | status | outer], double results [resid], P2, R2;
// img: the nine block images for the tensor-core engine, or null).
extern "C" cudaError_t bt_mrhs_solve_launch(int N, int n, int m, const double* alpha, const float* const* blk32,
                                            const double* D64, const double* O64, int bs32, int bs64,
                                            void* const* vec, const float* const* img, double tol, double tol_inner,
                                            int maxit, int max_outer, long long budget, int G, int nrhs,
                                            const double* B, double* X, int smem, cudaStream_t st) {
  bt::MParams P{};
  P.D32 = blk32[0]; P.O32 = blk32[1]; P.Dinv32 = blk32[2]; P.E32 = blk32[3];
  P.Hd32 = blk32[4]; P.Hu32 = blk32[5]; P.Hl32 = blk32[6];
  P.D64 = D64;
  P.O64 = O64;
  if (img) {
    P.img_d = img[0]; P.img_dinv = img[1]; P.img_hd = img[2];
    P.img_ot = img[3]; P.img_et = img[4]; P.img_hl = img[5];
    P.img_o = img[6]; P.img_e = img[7]; P.img_hu = img[8];
  }
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
  P.R2 = static_cast<float*>(vec[16]);
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
  return bt_launch_mrhs(&P, B, X, smem, img ? 1 : 0, st);
}
