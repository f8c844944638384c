// Shared definitions for the libbt CUDA sources (sm_103a).
//
// Library block layout.  Every block array (D, O, D^-1, E, Hd, Hu, Hl) holds,
// per instance, N slots of `bs` elements, one slot per block row i (the
// arrays with fewer real blocks -- O and E have N-1, Hu and Hl have N-2 --
// keep zero-filled padding slots so that every array indexes by row).  `bs`
// is n*n rounded up to 16 bytes so that each block starts on the 16-byte
// boundary a bulk copy needs.  Inside a slot the block is stored
// column-major: element (a, c) at c*n + a.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace bt {

constexpr int kMaxM = 8;
constexpr int kMaxBlock = 64;
constexpr int kMaxStages = 8;
#ifndef BT_THREADS
#define BT_THREADS 256
#endif
#ifndef BT_LEADER_WARP
#define BT_LEADER_WARP (BT_THREADS / 32 - 1)
#endif
constexpr int kThreads = BT_THREADS;    // threads per persistent CTA
// Thread that issues the bulk copies: lane 0 of the last warp.  Per-chunk
// work is spread from thread 0 upwards, so the last warp is the idlest one
// and the copy issue stays off the chunk's critical path.
constexpr int kLeaderTid = 32 * BT_LEADER_WARP;
constexpr int kMaxChunkElems = 512;     // rows-per-chunk cap: R * n <= 512

enum Status : int {
  kOK = 0, kErrArg = 1, kErrParam = 2, kErrNotSPD = 3, kErrNoConv = 4,
  kErrBreakdown = 5, kErrNonfinite = 6, kErrTimeout = 7
};

struct InstDesc {
  int N, n;
  int bs32, bs64;          // padded block stride in elements
  long long off32, off64;  // element offset of block row 0 in every block array
  long long vec;           // element offset of the instance's vectors in b / x
};

enum Op : int { kOpSolve = 0, kOpSpmv64 = 1, kOpSpmv32 = 2, kOpApply = 3 };

struct KParams {
  const double *D64, *O64, *Dinv64, *E64, *Hd64, *Hu64, *Hl64;
  const float *D32, *O32, *Dinv32, *E32, *Hd32, *Hu32, *Hl32;
  // general member of the family (a < 1): the +-1 blocks of H_ab,
  // F_i = -(1-a) D_i^-1 O_i and K_i = -(1-a) D_{i+1}^-1 O_i^T (slot i, i < N-1)
  const double *F64, *K64;
  const float *F32, *K32;
  double* hist;            // optional [B][hist_len][3]: per PCG iteration k the relative
  int hist_len;            // residual of its inner solve, alpha_k and beta_k (null = off)
  int variant;             // kernel: 0 optimum (stored H_opt), 1 general member
                           // (five-array H_ab), 2 optimum with the matrix-free H_opt
  const InstDesc* inst;
  const int* order;        // instance processing order (largest first)
  int B;
  int* queue;              // work counter, zeroed before launch
  const double* bvec;      // SOLVE: b;  SPMV: x;  APPLY: r
  double* xvec;            // SOLVE: x;  SPMV: y;  APPLY: z
  int op, mixed, m;
  int scal64;              // mixed: divide the inner CG step scalars in float64 (else float32)
  double alpha[kMaxM];
  double tol, tol_inner;
  int maxit, max_outer, use_x0;
  long long budget;        // clock cycles per instance solve
  char* ws;                // workspace: one slot per CTA (batched) or one shared slot
  long long ws_stride;     // bytes per slot
  long long ws_vec;        // elements per vector in a slot (>= max N*n)
  int G;                   // CTAs per instance (1 = batched mode)
  unsigned* bar;           // group barrier counter (zeroed before launch)
  double* red;             // group reduction slots [2][G][4]
  int* abort_flag;
  int* iters; int* status; int* outer; double* resid; double* errval;
  int stages, stage_bytes;
  int vec_slot_bytes;      // bytes of one vector-ring slot
};

// Per-thread dot-product partials: float32 products summed with a compensated
// float32 sum (TwoSum: each addition's rounding error is carried in c, so the
// partial stays within a few float32 ulps whatever the number of terms),
// widened to float64 once; float64 partials sum plainly.
template <typename T>
struct Accum;
template <>
struct Accum<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    const float bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};
template <>
struct Accum<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};

// Slot stride (in floats) of a float32 n x n block in the library layout.
// A multiple of 4 (16-byte aligned slots for bulk copies); for n % 4 == 0 also
// congruent to n modulo 32, so that consecutive blocks continue the bank
// sequence of one column-major matrix: a warp whose lanes read column c of two
// neighbouring blocks touches 32 consecutive banks (no shared-memory bank
// conflicts in the chunk products) at the price of <= 31 padding floats.
__host__ __device__ inline int slot32(int n) {
  int s = (n * n + 3) / 4 * 4;
  if (n % 4 == 0)
    while (s % 32 != n % 32) s += 4;
  return s;
}

struct RowRef {
  int inst, row;
};
struct SegRef {  // block rows [a, b) of one instance
  int inst, a, b, pad;
};

struct SetupParams {
  const InstDesc* inst;
  const RowRef* rows;
  long long nrows;
  const double* D;          // caller's D (row-major blocks)
  const double* O;          // caller's O
  const long long* d_off;   // per instance, element offsets in D / O
  const long long* o_off;
  double *D64, *O64, *Dinv64, *E64, *Hd64, *Hu64, *Hl64;
  float *D32, *O32, *Dinv32, *E32, *Hd32, *Hu32, *Hl32;
  double *F64, *K64;        // general member only (fam_a < 1), else null
  float *F32, *K32;
  double fam_a;             // multi-splitting weight a (1 = the optimum)
  int want32, want64;       // which precisions to produce
  unsigned long long* fail_key;  // min over failing (inst << 32 | row)
  double* fail_piv;         // per global row: the failing pivot
  int* retry;               // mixed only, optional: [0] = count, [1..] = rows whose
                            // float32 factor was refused (refactored in float64)
  const SegRef* segs;       // mixed only, optional: row segments for the fused E/H kernel
  long long nsegs;
  int copied;               // mixed: D64, O64, D32, O32 already hold the blocks (written by the
                            // LQR formation); the factor reads D from them and copies nothing
  // mixed, optional: canonical row indices grouped by block-size class
  // (0: n = 12, 1: 24, 2: 36, 3: any other n), class c at [cls_lo[c], cls_hi[c]);
  // null: one float32 factor kernel over all rows
  const long long* cls_idx;
  long long cls_lo[4], cls_hi[4];
  long long seg_lo[4], seg_hi[4];  // with cls_idx: the segments of each class, grouped in segs
};

struct AdjParams {
  const InstDesc* inst;
  const RowRef* rows;
  long long nrows;
  const long long* d_off;
  const long long* o_off;
  const double* x;
  const double* g;
  double* gD;
  double* gO;
};


// ---------------------------------------------------------------------------
// PTX helpers: mbarrier, bulk global->shared copy through the TMA engine.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Order this thread's earlier generic-proxy global writes before later
// async-proxy (bulk copy) reads of the same addresses.
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: returns false if `deadline` (clock64 cycles) passes first.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity, long long deadline) {
  while (!mbar_try_wait(b, parity)) {
    if (clock64() > deadline) return false;
  }
  return true;
}

// bytes must be a multiple of 16; both addresses 16-byte aligned.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(b))
      : "memory");
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_volatile_i32(const int* p) {
  return *reinterpret_cast<const volatile int*>(p);
}

// floor(t / d) for 0 <= t < 16384 and 1 <= d <= 64 without an integer divide:
// (t + 1/2) / d is at least 1/(2d) away from an integer, far more than the
// float rounding error at these sizes.
__device__ __forceinline__ int qdiv(int t, float inv_d) {
  return __float2int_rz(__fmul_rn(__int2float_rn(t) + 0.5f, inv_d));
}

template <typename T>
__device__ __forceinline__ bool is_finite(T v) {
  return isfinite(v);
}

}  // namespace bt
