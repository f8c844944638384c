// Setup kernels: the preconditioner blocks of Sec. 4.1 for every block row of
// every instance, plus the layout copies of D and O, and the adjoint's block
// outer products.
//
//   K1  (one warp per block row) copy D_i, O_i (row-major, caller's) into the
//       library layout (column-major, 16-byte padded slots) in float64 and/or
//       float32; D_i = L_i L_i^T by Cholesky in float64, W = L_i^-1,
//       D_i^-1 = W^T W (float64 for the float64 handle; float32 from the
//       float64 factor for the mixed handle)
//   K2  E_i = D_i^-1 O_i D_{i+1}^-1
//   K3  Hd_i = E_{i-1}^T O_{i-1} + E_i O_i^T, Hu_i = E_i O_{i+1},
//       Hl_i = E_{i+1}^T O_i^T          (only for polynomial order m >= 2)
// K2, K3: one CTA per block row; block products out of shared memory with
// 4 x 4 register tiles.
#include <algorithm>

#include "bt_common.cuh"

namespace bt {

// ---------------------------------------------------------------- K0+K1
// One warp per block row: load D_i (and O_i) once, write the library copies
// (column-major; float64 and, for mixed handles, float32), factor D_i by
// Cholesky in float64, invert the factor and form D_i^-1 = W^T W in MT.
// Warp-synchronous: no CTA barriers, so a CTA hosts several block rows.
template <typename MT>
__device__ void factor_row64(const SetupParams& P, long long gr, char* wsm) {
  const int lane = threadIdx.x & 31;
  const RowRef rr = P.rows[gr];
  const InstDesc d = P.inst[rr.inst];
  const int n = d.n, i = rr.row, nn = n * n;
  double* A = reinterpret_cast<double*>(wsm);  // 16 maxn^2 + 512 bytes per warp
  double* T = A + nn;
  // the caller's D (row-major), or with P.copied the library's float64 copy
  // (column-major: the same array for a symmetric D)
  const double* Du = P.copied ? P.D64 + d.off64 + (long long)i * d.bs64 : P.D + P.d_off[rr.inst] + (long long)i * nn;
  const bool hasO = i < d.N - 1;
  for (int t = lane; t < nn; t += 32) A[t] = Du[t];
  if (hasO && !P.copied) {
    const double* Ou = P.O + P.o_off[rr.inst] + (long long)i * nn;
    for (int t = lane; t < nn; t += 32) T[t] = Ou[t];
  }
  __syncwarp();
  const float inv_n = 1.0f / (float)n;
  if (!P.copied) {
    double* D64 = P.D64 + d.off64 + (long long)i * d.bs64;
    double* O64 = P.O64 + d.off64 + (long long)i * d.bs64;
    float* D32 = P.want32 ? P.D32 + d.off32 + (long long)i * d.bs32 : nullptr;
    float* O32 = P.want32 ? P.O32 + d.off32 + (long long)i * d.bs32 : nullptr;
    for (int t = lane; t < nn; t += 32) {  // destination column-major index t = c*n + a
      const int c = qdiv(t, inv_n), a = t - c * n;
      const double dv = A[a * n + c];
      D64[t] = dv;
      if (D32) D32[t] = (float)dv;
      if (hasO) {
        const double ov = T[a * n + c];
        O64[t] = ov;
        if (O32) O32[t] = (float)ov;
      }
    }
  }
  __syncwarp();
  // Cholesky D = L L^T in place (lower triangle of A, row-major), float64.
  // Float64 runs at 1/58 of the float32 rate here, so every float64
  // warp-instruction counts: one rsqrt per column gives both the pivot
  // (piv * rsqrt(piv)) and its reciprocal, and the trailing update walks
  // only the lower triangle (triangular index t -> (rr, cc), rr >= cc).
  double* rinv_col = T + nn;  // reciprocals of the diagonal of L (warp tail)
  for (int j = 0; j < n; ++j) {
    const double piv = A[j * n + j];
    if (!(piv > 0.0) || !isfinite(piv)) {
      if (lane == 0) {
        P.fail_piv[gr] = piv;
        atomicMin(P.fail_key, ((unsigned long long)rr.inst << 32) | (unsigned)i);
      }
      return;
    }
    const double rinv = rsqrt(piv);
    __syncwarp();
    for (int r = j + 1 + lane; r < n; r += 32) A[r * n + j] *= rinv;
    if (lane == 0) {
      A[j * n + j] = piv * rinv;
      rinv_col[j] = rinv;
    }
    __syncwarp();
    const int m = n - j - 1;
    const int tri = m * (m + 1) / 2;
    for (int t = lane; t < tri; t += 32) {
      int rq = __float2int_rz((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
      if ((rq + 1) * (rq + 2) / 2 <= t) ++rq;   // guard the float estimate
      if (rq * (rq + 1) / 2 > t) --rq;
      const int cq = t - rq * (rq + 1) / 2;
      const int r = j + 1 + rq, c = j + 1 + cq;
      A[r * n + c] = fma(-A[r * n + j], A[c * n + j], A[r * n + c]);
    }
    __syncwarp();
  }
  // W = L^-1 (one column per lane, forward substitution) and D_i^-1 = W^T W,
  // both in float64 (the reciprocals of the diagonal of L come from the
  // Cholesky); the result is rounded to MT once, on the store.
  double* W = T;
  const double* dv = rinv_col;
  for (int c = lane; c < n; c += 32) {
    for (int r = 0; r < c; ++r) W[r * n + c] = 0.0;
    W[c * n + c] = dv[c];
    for (int r = c + 1; r < n; ++r) {
      double acc = 0.0;
      for (int t = c; t < r; ++t) acc = fma(A[r * n + t], W[t * n + c], acc);
      W[r * n + c] = -acc * dv[r];
    }
  }
  __syncwarp();
  MT* out = (sizeof(MT) == 8) ? reinterpret_cast<MT*>(P.Dinv64 + d.off64 + (long long)i * d.bs64)
                              : reinterpret_cast<MT*>(P.Dinv32 + d.off32 + (long long)i * d.bs32);
  for (int t = lane; t < nn; t += 32) {
    const int a = qdiv(t, inv_n), b = t - a * n;
    if (a < b) continue;
    double acc = 0.0;
    for (int r = a; r < n; ++r) acc = fma(W[r * n + a], W[r * n + b], acc);
    out[(long long)b * n + a] = (MT)acc;
    out[(long long)a * n + b] = (MT)acc;
  }
}

template <typename MT>
__global__ void k_factor(const __grid_constant__ SetupParams P, int wpc, int warp_bytes) {
  extern __shared__ __align__(16) char smraw[];
  const int warp = threadIdx.x >> 5;
  const long long gr = (long long)blockIdx.x * wpc + warp;
  if (gr >= P.nrows) return;
  factor_row64<MT>(P, gr, smraw + (size_t)warp * warp_bytes);
}

// Float64 refactor of the rows whose float32 factor was refused (list in
// P.retry); a float64 failure here is the handle's NOT_SPD.
__global__ void k_factor_retry(const __grid_constant__ SetupParams P, int wpc, int warp_bytes) {
  extern __shared__ __align__(16) char smraw[];
  const int warp = threadIdx.x >> 5;
  const int count = *(volatile const int*)P.retry;
  for (long long k = (long long)blockIdx.x * wpc + warp; k < count; k += (long long)gridDim.x * wpc)
    factor_row64<float>(P, P.retry[1 + k], smraw + (size_t)warp * warp_bytes);
}

// ---------------------------------------------------------------- K1 (mixed), registers
// Register-resident float32 factor for compile-time block sizes: lane l owns
// rows (and, for W, columns) l and l + 32.  Cholesky right-looking by rows,
// W = L^-1 by columns (forward substitution), D^-1 = W^T W by columns; the
// operands another lane owns arrive by warp shuffle.  Returns false when a
// pivot is refused (same rule as the shared-memory path).  The upper parts of
// the row registers take harmless updates (each stays a finite combination of
// entries of D and L) and are never read.
template <int NB>
__device__ __forceinline__ bool factor_regs(const float* __restrict__ D32, float* __restrict__ out, int lane) {
  constexpr int H = (NB + 31) / 32;
  constexpr unsigned FULL = 0xffffffffu;
  float a[H][NB];
#pragma unroll
  for (int h = 0; h < H; ++h) {
    const int r = lane + 32 * h;
#pragma unroll
    for (int c = 0; c < NB; ++c) a[h][c] = (r < NB) ? __ldcg(D32 + c * NB + r) : 0.f;
  }
  float rown[H];  // 1 / L_rr of the lane's own rows
#pragma unroll
  for (int h = 0; h < H; ++h) rown[h] = 0.f;
  bool ok = true;  // a refused pivot is replaced by 1 and reported at the end
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    float piv = __shfl_sync(FULL, a[j / 32][j], j % 32);
    const float dj = __ldcg(D32 + j * NB + j);
    if (!(piv > 0.f && piv > 1e-3f * dj) || !(piv < INFINITY)) {
      ok = false;
      piv = 1.f;
    }
    const float ri = rsqrtf(piv);
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const int r = lane + 32 * h;
      a[h][j] = (r > j) ? a[h][j] * ri : ((r == j) ? piv * ri : a[h][j]);
      rown[h] = (r == j) ? ri : rown[h];
    }
#pragma unroll
    for (int c = 0; c < NB; ++c) {  // constant bounds: the compiler unrolls both loops
      if (c <= j) continue;
      const float lc = __shfl_sync(FULL, a[c / 32][j], c % 32);  // L(c, j)
#pragma unroll
      for (int h = 0; h < H; ++h) a[h][c] = fmaf(-a[h][j], lc, a[h][c]);
    }
  }
  if (!ok) return false;
  // W(r, c), lane column c = lane + 32 h: W(c, c) = 1/L_cc, zero above
  float w[H][NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    float acc0[H], acc1[H];
#pragma unroll
    for (int h = 0; h < H; ++h) acc0[h] = acc1[h] = 0.f;
#pragma unroll
    for (int t = 0; t < NB; ++t) {
      if (t >= r) continue;
      const float lrt = __shfl_sync(FULL, a[r / 32][t], r % 32);  // L(r, t)
#pragma unroll
      for (int h = 0; h < H; ++h) {
        if (t & 1) acc1[h] = fmaf(lrt, w[h][t], acc1[h]);
        else acc0[h] = fmaf(lrt, w[h][t], acc0[h]);
      }
    }
    const float dr = __shfl_sync(FULL, rown[r / 32], r % 32);  // 1 / L_rr
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const int c = lane + 32 * h;
      w[h][r] = (r > c) ? -(acc0[h] + acc1[h]) * dr : ((r == c) ? dr : 0.f);
    }
  }
  // D^-1(a, b) = sum_{r >= b} W(r, a) W(r, b) (terms with r < a vanish)
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    float acc0[H], acc1[H];
#pragma unroll
    for (int h = 0; h < H; ++h) acc0[h] = acc1[h] = 0.f;
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      if (r < b) continue;
      const float wrb = __shfl_sync(FULL, w[b / 32][r], b % 32);  // W(r, b)
#pragma unroll
      for (int h = 0; h < H; ++h) {
        if (r & 1) acc1[h] = fmaf(w[h][r], wrb, acc1[h]);
        else acc0[h] = fmaf(w[h][r], wrb, acc0[h]);
      }
    }
#pragma unroll
    for (int h = 0; h < H; ++h)
      if (lane + 32 * h < NB) out[b * NB + lane + 32 * h] = acc0[h] + acc1[h];
  }
  return true;
}

// ---------------------------------------------------------------- K1 (mixed)
// Float32 factor for mixed handles, one warp per block row in a 4 n (n+1)
// byte shared region (+ 64 floats):
//   1. D_i, O_i -> library copies (float64 and float32, column-major), staged
//      through shared memory half a block at a time;
//   2. D_i = L L^T by Cholesky in float32, column-major in place (lane = row);
//   3. W = L^-1 (lane = column), its strict lower part kept in the unused
//      upper triangle and its diagonal (1 / L_jj) in the 64-float tail;
//   4. D_i^-1 = W^T W, one column per step (lane = row), coalesced stores.
// A pivot below 1e-3 of its original diagonal means kappa(D_i) > 1e3 (the
// pivot is at least lambda_min, the diagonal at most lambda_max); such rows
// and non-positive or non-finite pivots go to the float64 retry list, so a
// poorly conditioned block costs float64 time only where it occurs.
// One row of k_factor32.  NB > 0: the register-resident factor for n = NB;
// 0: the register variant chosen at run time for n in {12, 24, 36}, the
// shared-memory walk otherwise; -1: the shared-memory walk only.  (A kernel
// holding only one variant takes that variant's registers, not the largest
// one's.)
template <int NB>
__device__ __forceinline__ void factor32_row(const SetupParams& P, long long gr, char* wsm, int warp_bytes,
                                             int lane) {
  const RowRef rr = P.rows[gr];
  const InstDesc d = P.inst[rr.inst];
  const int n = d.n, i = rr.row, nn = n * n;
  float* A = reinterpret_cast<float*>(wsm);
  float* dv = reinterpret_cast<float*>(wsm + warp_bytes - 64 * sizeof(float));
  double* stg = reinterpret_cast<double*>(wsm);
  float* D32 = P.D32 + d.off32 + (long long)i * d.bs32;
  // 1. layout copies: rows [a0, a0 + h) of the caller's row-major block
  const auto copy_block = [&](const double* src, double* dst64, float* dst32) {
    for (int a0 = 0; a0 < n; a0 += (n + 1) / 2) {
      const int h = min((n + 1) / 2, n - a0), cnt = h * n;
      const float inv_h = 1.0f / (float)h;
      // asynchronous 8-byte copies: every element of the half block in flight
      // at once instead of one global round trip per loop iteration
      for (int t = lane; t < cnt; t += 32)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(stg + t)),
                     "l"(src + (long long)a0 * n + t)
                     : "memory");
      asm volatile("cp.async.commit_group;" ::: "memory");
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      __syncwarp();
      for (int t = lane; t < cnt; t += 32) {  // t = c * h + (a - a0)
        const int c = qdiv(t, inv_h), ar = t - c * h;
        const double v = stg[ar * n + c];
        dst64[(long long)c * n + a0 + ar] = v;
        dst32[(long long)c * n + a0 + ar] = (float)v;
      }
      __syncwarp();
    }
  };
  if (!P.copied) {
    if (i < d.N - 1)
      copy_block(P.O + P.o_off[rr.inst] + (long long)i * nn, P.O64 + d.off64 + (long long)i * d.bs64,
                 P.O32 + d.off32 + (long long)i * d.bs32);
    copy_block(P.D + P.d_off[rr.inst] + (long long)i * nn, P.D64 + d.off64 + (long long)i * d.bs64, D32);
  }
  float* out = P.Dinv32 + d.off32 + (long long)i * d.bs32;
  {
    int done = -1;  // -1: no register variant for this n
    if constexpr (NB > 0) {
      done = factor_regs<NB>(D32, out, lane) ? 1 : 0;
    } else if constexpr (NB == 0) {
      switch (n) {
        case 12: done = factor_regs<12>(D32, out, lane) ? 1 : 0; break;
        case 24: done = factor_regs<24>(D32, out, lane) ? 1 : 0; break;
        case 36: done = factor_regs<36>(D32, out, lane) ? 1 : 0; break;
        default: break;
      }
    }
    if (done == 0 && lane == 0) P.retry[1 + atomicAdd(P.retry, 1)] = (int)gr;
    if (done >= 0) return;
  }
  // this warp's own float32 copy, column-major: A[c n + r] = D(r, c)
  for (int t = lane; t < nn; t += 32) A[t] = __ldcg(D32 + t);
  __syncwarp();
  for (int r = lane; r < n; r += 32) dv[r] = A[r * n + r];
  __syncwarp();
  // 2. Cholesky, lane owns rows r0 = lane and r1 = lane + 32
  const int r0 = lane, r1 = lane + 32;
  for (int j = 0; j < n; ++j) {
    const float piv = A[j * n + j];
    const float dj = dv[j];
    if (!(piv > 0.f && piv > 1e-3f * dj) || !(piv < INFINITY)) {
      if (lane == 0) P.retry[1 + atomicAdd(P.retry, 1)] = (int)gr;
      return;
    }
    const float rinv = rsqrtf(piv);
    __syncwarp();
    if (r0 > j && r0 < n) A[j * n + r0] *= rinv;
    if (r1 > j && r1 < n) A[j * n + r1] *= rinv;
    if (lane == 0) {
      A[j * n + j] = piv * rinv;
      dv[j] = rinv;
    }
    __syncwarp();
    const float l0 = (r0 > j && r0 < n) ? A[j * n + r0] : 0.f;
    const float l1 = (r1 > j && r1 < n) ? A[j * n + r1] : 0.f;
    for (int c = j + 1; c < n; ++c) {
      const float bc = A[j * n + c];
      if (c <= r0 && r0 < n) A[c * n + r0] = fmaf(-l0, bc, A[c * n + r0]);
      if (c <= r1 && r1 < n) A[c * n + r1] = fmaf(-l1, bc, A[c * n + r1]);
    }
    __syncwarp();
  }
  // 3. W = L^-1: W(r, c) = -(1/L_rr) sum_{t=c}^{r-1} L(r, t) W(t, c), with
  //    L(r, t) = A[t n + r], W(t, c) = A[t n + c] for t > c, W(c, c) = dv[c]
  for (int c = lane; c < n; c += 32) {
    const float wcc = dv[c];
    for (int r = c + 1; r < n; ++r) {
      float acc = A[c * n + r] * wcc;
      for (int t = c + 1; t < r; ++t) acc = fmaf(A[t * n + r], A[t * n + c], acc);
      A[r * n + c] = -acc * dv[r];
    }
  }
  __syncwarp();
  // 4. D_i^-1(a, b) = sum_{r >= max(a, b)} W(r, a) W(r, b), column b per step
  for (int b = 0; b < n; ++b) {
    float acc0 = 0.f, acc1 = 0.f;
    for (int r = b; r < n; ++r) {
      const float wrb = (r == b) ? dv[b] : A[r * n + b];
      const float w0 = (r > r0) ? A[r * n + r0] : (r == r0 ? dv[r0] : 0.f);
      acc0 = fmaf(w0, wrb, acc0);
      if (n > 32) {
        const float w1 = (r > r1) ? A[r * n + r1] : (r == r1 ? dv[r1 & 63] : 0.f);
        acc1 = fmaf(w1, wrb, acc1);
      }
    }
    if (r0 < n) out[(long long)b * n + r0] = acc0;
    if (r1 < n) out[(long long)b * n + r1] = acc1;
  }
}

__global__ void k_factor32(const __grid_constant__ SetupParams P, int wpc, int warp_bytes) {
  extern __shared__ __align__(16) char smraw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long gr = (long long)blockIdx.x * wpc + warp;
  if (gr >= P.nrows) return;
  factor32_row<0>(P, gr, smraw + (size_t)warp * warp_bytes, warp_bytes, lane);
}

// The rows of one block-size class (P.cls_idx[P.cls_lo[cls] ..
// P.cls_hi[cls]), canonical row indices), with that class's variant only.
template <int NB>
__global__ void k_factor32_cls(const __grid_constant__ SetupParams P, int wpc, int warp_bytes, int cls) {
  extern __shared__ __align__(16) char smraw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long li = P.cls_lo[cls] + (long long)blockIdx.x * wpc + warp;
  if (li >= P.cls_hi[cls]) return;
  factor32_row<NB>(P, P.cls_idx[li], smraw + (size_t)warp * warp_bytes, warp_bytes, lane);
}

// Small dense products in shared memory: matrices are row-major n x n.
// C (+)= op(A) op(B)
template <typename MT>
__device__ void sm_gemm(MT* C, const MT* A, bool tA, const MT* B, bool tB, int n, bool accumulate) {
  const float inv_n = 1.0f / (float)n;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int a = qdiv(t, inv_n), b = t - a * n;
    MT acc = accumulate ? C[t] : MT(0);
    for (int c = 0; c < n; ++c) {
      const MT av = tA ? A[c * n + a] : A[a * n + c];
      const MT bv = tB ? B[b * n + c] : B[c * n + b];
      acc = fma(av, bv, acc);
    }
    C[t] = acc;
  }
}

// 4 x 4 register tiles when n % 4 == 0 (else the plain loop above).
template <typename MT>
__device__ void sm_gemm4(MT* C, const MT* A, bool tA, const MT* B, bool tB, int n, bool accumulate) {
  if (n % 4 != 0) {
    sm_gemm(C, A, tA, B, tB, n, accumulate);
    return;
  }
  const int q = n / 4;
  const float inv_q = 1.0f / (float)q;
  for (int t = threadIdx.x; t < q * q; t += blockDim.x) {
    const int tq = qdiv(t, inv_q);
    const int a0 = tq * 4, b0 = (t - tq * q) * 4;
    MT acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = accumulate ? C[(a0 + r) * n + b0 + c] : MT(0);
    for (int k = 0; k < n; ++k) {
      MT av[4], bv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) av[r] = tA ? A[k * n + a0 + r] : A[(a0 + r) * n + k];
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[c] = tB ? B[(b0 + c) * n + k] : B[k * n + b0 + c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) C[(a0 + r) * n + b0 + c] = acc[r][c];
  }
}

// load a column-major library block into row-major shared memory
template <typename MT>
__device__ void sm_load(MT* dst, const MT* src, int n) {
  const float inv_n = 1.0f / (float)n;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {  // coalesced read of the column-major block
    const int c = qdiv(t, inv_n), a = t - c * n;
    dst[a * n + c] = src[t];
  }
}
template <typename MT>
__device__ void sm_store(MT* dst, const MT* src, int n) {
  const float inv_n = 1.0f / (float)n;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {  // coalesced write of the column-major block
    const int c = qdiv(t, inv_n), a = t - c * n;
    dst[t] = src[a * n + c];
  }
}

template <typename MT>
struct MatSet {
  const MT *O, *Dinv;
  MT *E, *Hd, *Hu, *Hl;
  long long off;
  int bs;
};

template <typename MT>
__device__ MatSet<MT> matset(const SetupParams& P, const InstDesc& d) {
  MatSet<MT> s;
  if (sizeof(MT) == 8) {
    s.O = (const MT*)P.O64; s.Dinv = (const MT*)P.Dinv64; s.E = (MT*)P.E64;
    s.Hd = (MT*)P.Hd64; s.Hu = (MT*)P.Hu64; s.Hl = (MT*)P.Hl64; s.off = d.off64; s.bs = d.bs64;
  } else {
    s.O = (const MT*)P.O32; s.Dinv = (const MT*)P.Dinv32; s.E = (MT*)P.E32;
    s.Hd = (MT*)P.Hd32; s.Hu = (MT*)P.Hu32; s.Hl = (MT*)P.Hl32; s.off = d.off32; s.bs = d.bs32;
  }
  return s;
}

// ---------------------------------------------------------------- K2
template <typename MT>
__global__ void k_E(const __grid_constant__ SetupParams P) {
  extern __shared__ __align__(16) char smraw[];
  const long long gr = blockIdx.x;
  if (gr >= P.nrows) return;
  const RowRef rr = P.rows[gr];
  const InstDesc d = P.inst[rr.inst];
  const int n = d.n, i = rr.row;
  if (i >= d.N - 1) return;  // padding slot stays zero
  MatSet<MT> M = matset<MT>(P, d);
  MT* s0 = reinterpret_cast<MT*>(smraw);
  MT* s1 = s0 + n * n;
  MT* s2 = s1 + n * n;
  const auto blk = [&](const MT* base, int row) { return base + M.off + (long long)row * M.bs; };
  sm_load(s0, blk(M.O, i), n);
  sm_load(s1, blk(M.Dinv, i + 1), n);
  __syncthreads();
  sm_gemm4(s2, s0, false, s1, false, n, false);  // T = O_i D_{i+1}^-1
  __syncthreads();
  sm_load(s0, blk(M.Dinv, i), n);
  __syncthreads();
  sm_gemm4(s1, s0, false, s2, false, n, false);  // E_i = D_i^-1 T
  __syncthreads();
  sm_store(const_cast<MT*>(blk(M.E, i)), s1, n);
}

// ---------------------------------------------------------------- K3
template <typename MT>
__global__ void k_H(const __grid_constant__ SetupParams P) {
  extern __shared__ __align__(16) char smraw[];
  const long long gr = blockIdx.x;
  if (gr >= P.nrows) return;
  const RowRef rr = P.rows[gr];
  const InstDesc d = P.inst[rr.inst];
  const int n = d.n, i = rr.row, N = d.N;
  MatSet<MT> M = matset<MT>(P, d);
  MT* sa = reinterpret_cast<MT*>(smraw);
  MT* sb = sa + n * n;
  MT* sc = sb + n * n;
  const auto blk = [&](const MT* base, int row) { return base + M.off + (long long)row * M.bs; };
  // Hd_i = E_{i-1}^T O_{i-1} + E_i O_i^T
  bool acc = false;
  if (i > 0) {
    sm_load(sa, blk(M.E, i - 1), n);
    sm_load(sb, blk(M.O, i - 1), n);
    __syncthreads();
    sm_gemm4(sc, sa, true, sb, false, n, false);
    acc = true;
    __syncthreads();
  }
  if (i < N - 1) {
    sm_load(sa, blk(M.E, i), n);
    sm_load(sb, blk(M.O, i), n);
    __syncthreads();
    sm_gemm4(sc, sa, false, sb, true, n, acc);
    acc = true;
    __syncthreads();
  }
  if (acc) sm_store(const_cast<MT*>(blk(M.Hd, i)), sc, n);
  __syncthreads();
  if (i < N - 2) {
    // Hu_i = E_i O_{i+1}
    sm_load(sa, blk(M.E, i), n);
    sm_load(sb, blk(M.O, i + 1), n);
    __syncthreads();
    sm_gemm4(sc, sa, false, sb, false, n, false);
    __syncthreads();
    sm_store(const_cast<MT*>(blk(M.Hu, i)), sc, n);
    __syncthreads();
    // Hl_i = E_{i+1}^T O_i^T
    sm_load(sa, blk(M.E, i + 1), n);
    sm_load(sb, blk(M.O, i), n);
    __syncthreads();
    sm_gemm4(sc, sa, true, sb, true, n, false);
    __syncthreads();
    sm_store(const_cast<MT*>(blk(M.Hl, i)), sc, n);
  }
}

// ---------------------------------------------------------------- K4
// The general member (a, b = 1 - 2a) of the family, a < 1.  With the block
// Jacobi iteration matrix H_J = B_d^-1 C_d, the multi-splitting of Sec. 3.1
// gives G_ab = B_d^-1 + a B_d^-1 C_d B_d^-1 and H_ab = (1 - a) H_J + a H_J^2;
// C_d is minus the off-diagonal part of S, so B_d^-1 C_d B_d^-1 has the
// blocks -E_i, -E_i^T and H_J^2 has the pentadiagonal blocks of H_opt
// (Sec. 4.1).  This kernel therefore scales the stored E, Hd, Hu, Hl of row
// i by a, and forms the +-1 blocks of H_ab that H_opt lacks:
//     F_i = -(1 - a) D_i^-1 O_i          (block (i, i+1))
//     K_i = -(1 - a) D_{i+1}^-1 O_i^T    (block (i+1, i), kept in slot i)
template <typename MT>
__global__ void k_FK(const __grid_constant__ SetupParams P) {
  extern __shared__ __align__(16) char smraw[];
  const long long gr = blockIdx.x;
  if (gr >= P.nrows) return;
  const RowRef rr = P.rows[gr];
  const InstDesc d = P.inst[rr.inst];
  const int n = d.n, i = rr.row, N = d.N;
  MatSet<MT> M = matset<MT>(P, d);
  MT* F = (sizeof(MT) == 8) ? (MT*)P.F64 : (MT*)P.F32;
  MT* K = (sizeof(MT) == 8) ? (MT*)P.K64 : (MT*)P.K32;
  const MT wa = (MT)P.fam_a, wc = (MT)(-(1.0 - P.fam_a));
  const long long o = M.off + (long long)i * M.bs;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    if (i < N - 1) M.E[o + t] *= wa;
    if (M.Hd) {
      M.Hd[o + t] *= wa;
      if (i < N - 2) {
        M.Hu[o + t] *= wa;
        M.Hl[o + t] *= wa;
      }
    }
  }
  if (i >= N - 1 || !F) return;  // padding slots stay zero
  MT* s0 = reinterpret_cast<MT*>(smraw);
  MT* s1 = s0 + n * n;
  MT* s2 = s1 + n * n;
  const auto blk = [&](const MT* base, int row) { return base + M.off + (long long)row * M.bs; };
  const float inv_n = 1.0f / (float)n;
  const auto store_scaled = [&](MT* dst) {  // row-major smem -> column-major slot, times wc
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
      const int c = qdiv(t, inv_n), a = t - c * n;
      dst[t] = wc * s2[a * n + c];
    }
  };
  sm_load(s0, blk(M.Dinv, i), n);
  sm_load(s1, blk(M.O, i), n);
  __syncthreads();
  sm_gemm4(s2, s0, false, s1, false, n, false);  // D_i^-1 O_i
  __syncthreads();
  store_scaled(F + o);
  sm_load(s0, blk(M.Dinv, i + 1), n);
  __syncthreads();
  sm_gemm4(s2, s0, false, s1, true, n, false);   // D_{i+1}^-1 O_i^T
  __syncthreads();
  store_scaled(K + o);
}

// ---------------------------------------------------------------- K2+K3 (mixed)
// E and H fused over a segment of consecutive block rows [a, b) of one
// instance, all blocks column-major float32 in shared-memory rings.  Step j
// (j = a-2 .. b+1) forms, as independent tile tasks,
//   T_{j+1} = O_{j+1} D_{j+2}^-1            (kept for the next step)
//   E_j     = D_j^-1 T_j                    (rows a-1 .. b; stored for j in [a, b))
//   H_{j-2}: Hd = E^T_{i-1} O_{i-1} + E_i O_i^T, Hu = E_i O_{i+1},
//            Hl = E_{i+1}^T O_i^T           (i = j-2 in [a, b))
// while cp.async prefetches O_{j+2} and D_{j+3}^-1 for the next step.  E_j is
// also kept transposed, so that every product reads its left operand along a
// column (no strided shared-memory reads).  Ring sizes follow the block
// lifetimes: O 6, D^-1 4, T 2, E 4, E^T 4 slots.  Every output element is one
// fma chain over k = 0 .. n-1 (two chains in a row for Hd), the same
// arithmetic as K2/K3.
constexpr int kEHSlots = 20;

// acc(r, c) += sum_k A(a0 + r, k) opB(k, b0 + c); X(a, c) at X[c n + a];
// TB: opB = B^T.
template <int TS, bool TB>
__device__ __forceinline__ void tile_acc(float (&acc)[TS][TS], const float* __restrict__ A,
                                         const float* __restrict__ B, int n, int a0, int b0) {
  if constexpr (TS == 4) {  // n % 4 == 0: 4-deep k steps, 128-bit loads of both operands
    for (int k = 0; k < n; k += 4) {
      float4 av[4], bv[4];
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) av[kk] = *reinterpret_cast<const float4*>(A + (k + kk) * n + a0);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        bv[q] = TB ? *reinterpret_cast<const float4*>(B + (k + q) * n + b0)     // row k+q of B^T: b0..b0+3
                   : *reinterpret_cast<const float4*>(B + (b0 + q) * n + k);    // column b0+q of B: k..k+3
      const float* af = reinterpret_cast<const float*>(av);
      const float* bf = reinterpret_cast<const float*>(bv);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float bkc = TB ? bf[kk * 4 + c] : bf[c * 4 + kk];
            acc[r][c] = fmaf(af[kk * 4 + r], bkc, acc[r][c]);
          }
    }
  } else {
    for (int k = 0; k < n; ++k) {
      float av[TS], bv[TS];
#pragma unroll
      for (int r = 0; r < TS; ++r) av[r] = A[k * n + a0 + r];
#pragma unroll
      for (int c = 0; c < TS; ++c) bv[c] = TB ? B[k * n + b0 + c] : B[(b0 + c) * n + k];
#pragma unroll
      for (int r = 0; r < TS; ++r)
#pragma unroll
        for (int c = 0; c < TS; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
    }
  }
}

// C(a0 + r, b0 + c) = acc(r, c); TR: store C^T instead.
template <int TS, bool TR = false>
__device__ __forceinline__ void tile_store(float* C, const float (&acc)[TS][TS], int n, int a0, int b0) {
  if constexpr (TS == 4) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if constexpr (TR)
        *reinterpret_cast<float4*>(C + (a0 + q) * n + b0) = make_float4(acc[q][0], acc[q][1], acc[q][2], acc[q][3]);
      else
        *reinterpret_cast<float4*>(C + (b0 + q) * n + a0) = make_float4(acc[0][q], acc[1][q], acc[2][q], acc[3][q]);
    }
  } else {
#pragma unroll
    for (int c = 0; c < TS; ++c)
#pragma unroll
      for (int r = 0; r < TS; ++r) {
        if constexpr (TR) C[(a0 + r) * n + b0 + c] = acc[r][c];
        else C[(b0 + c) * n + a0 + r] = acc[r][c];
      }
  }
}

__device__ __forceinline__ void cp16(void* smem, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(smem)), "l"(g)
               : "memory");
}

template <int TS>
__device__ void eh_segment(const SetupParams& P, const SegRef sg, bool want_h, float* fsm) {
  const InstDesc d = P.inst[sg.inst];
  const int n = d.n, N = d.N, a = sg.a, b = sg.b, bs = d.bs32;
  const float* Og = P.O32 + d.off32;
  const float* Dg = P.Dinv32 + d.off32;
  float* Eg = P.E32 + d.off32;
  float* sO = fsm;
  float* sD = sO + 6 * bs;
  float* sT = sD + 4 * bs;
  float* sE = sT + 2 * bs;
  float* sET = sE + 4 * bs;
  // slot of block k (k >= -3 here, so k + 12 > 0)
  const auto O_ = [&](int k) { return sO + ((k + 12) % 6) * bs; };
  const auto D_ = [&](int k) { return sD + ((k + 12) % 4) * bs; };
  const auto T_ = [&](int k) { return sT + ((k + 12) % 2) * bs; };
  const auto E_ = [&](int k) { return sE + ((k + 12) % 4) * bs; };
  const auto ET_ = [&](int k) { return sET + ((k + 12) % 4) * bs; };
  const auto load = [&](float* dst, const float* src) {
    for (int t = threadIdx.x * 4; t < bs; t += blockDim.x * 4) cp16(dst + t, src + t);
  };
  // O_k is read up to k = b, D_k^-1 up to k = b + 1
  const auto wantO = [&](int k) { return k >= 0 && k <= N - 2 && k >= a - 1 && k <= b; };
  const auto wantD = [&](int k) { return k >= 0 && k <= N - 1 && k >= a - 1 && k <= b + 1; };
  if (wantO(a - 1)) load(O_(a - 1), Og + (long long)(a - 1) * bs);
  if (wantD(a - 1)) load(D_(a - 1), Dg + (long long)(a - 1) * bs);
  if (wantD(a)) load(D_(a), Dg + (long long)a * bs);
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  const int q = n / TS, tq = q * q;
  const float inv_q = 1.0f / (float)q;
  for (int j = a - 2; j <= b + 1; ++j) {
    if (wantO(j + 2)) load(O_(j + 2), Og + (long long)(j + 2) * bs);
    if (wantD(j + 3)) load(D_(j + 3), Dg + (long long)(j + 3) * bs);
    asm volatile("cp.async.commit_group;" ::: "memory");
    const int i = j - 2;
    const bool doT = (j + 1 >= 0) && (j + 1 <= N - 2) && (j + 1 >= a - 1) && (j + 1 <= b);
    const bool doE = (j >= 0) && (j <= N - 2) && (j >= a - 1) && (j <= b);
    const bool doH = want_h && i >= a && i < b;
    const bool doHd = doH && (i > 0 || i < N - 1);
    const bool doHu = doH && i <= N - 3;
    const unsigned mask = (doT ? 1u : 0u) | (doE ? 2u : 0u) | (doHd ? 4u : 0u) | (doHu ? 24u : 0u);
    const int njobs = __popc(mask);
    for (int idx = threadIdx.x; idx < njobs * tq; idx += blockDim.x) {
      const int js = idx / tq;
      const int tile = idx - js * tq;
      // job = position of the (js+1)-th set bit of mask
      unsigned mm = mask;
      for (int t = 0; t < js; ++t) mm &= mm - 1;
      const int job = __ffs(mm) - 1;
      const int tb = qdiv(tile, inv_q), ta = tile - tb * q;
      const int a0 = ta * TS, b0 = tb * TS;
      float acc[TS][TS];
#pragma unroll
      for (int r = 0; r < TS; ++r)
#pragma unroll
        for (int c = 0; c < TS; ++c) acc[r][c] = 0.f;
      if (job == 0) {
        tile_acc<TS, false>(acc, O_(j + 1), D_(j + 2), n, a0, b0);
        tile_store<TS>(T_(j + 1), acc, n, a0, b0);
      } else if (job == 1) {
        tile_acc<TS, false>(acc, D_(j), T_(j), n, a0, b0);
        tile_store<TS>(E_(j), acc, n, a0, b0);
        tile_store<TS, true>(ET_(j), acc, n, a0, b0);
        if (j >= a && j < b) tile_store<TS>(Eg + (long long)j * bs, acc, n, a0, b0);
      } else if (job == 2) {
        if (i > 0) tile_acc<TS, false>(acc, ET_(i - 1), O_(i - 1), n, a0, b0);
        if (i < N - 1) tile_acc<TS, true>(acc, E_(i), O_(i), n, a0, b0);
        tile_store<TS>(P.Hd32 + d.off32 + (long long)i * bs, acc, n, a0, b0);
      } else if (job == 3) {
        tile_acc<TS, false>(acc, E_(i), O_(i + 1), n, a0, b0);
        tile_store<TS>(P.Hu32 + d.off32 + (long long)i * bs, acc, n, a0, b0);
      } else {
        tile_acc<TS, true>(acc, ET_(i + 1), O_(i), n, a0, b0);
        tile_store<TS>(P.Hl32 + d.off32 + (long long)i * bs, acc, n, a0, b0);
      }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256, 2) k_EH(const __grid_constant__ SetupParams P, int want_h) {
  extern __shared__ __align__(16) float fsm[];
  const SegRef sg = P.segs[blockIdx.x];
  const int n = P.inst[sg.inst].n;
  if ((n & 3) == 0 && n >= 24) eh_segment<4>(P, sg, want_h != 0, fsm);
  else if ((n & 1) == 0) eh_segment<2>(P, sg, want_h != 0, fsm);
  else eh_segment<1>(P, sg, want_h != 0, fsm);
}

// The segments of one block-size class (segments [P.seg_lo[cls],
// P.seg_hi[cls]), grouped by class on the host) with one tile size: TS > 0
// that tile, 0 the choice by n as in k_EH.  Each kernel takes its own
// variant's registers and its class's shared memory; MINB CTAs per SM
// (n = 12 and 24: four, their rings are small enough).
template <int TS, int MINB>
__global__ void __launch_bounds__(256, MINB) k_EH_cls(const __grid_constant__ SetupParams P, int want_h, int cls) {
  extern __shared__ __align__(16) float fsm[];
  const SegRef sg = P.segs[P.seg_lo[cls] + blockIdx.x];
  if constexpr (TS > 0) {
    eh_segment<TS>(P, sg, want_h != 0, fsm);
  } else {
    const int n = P.inst[sg.inst].n;
    if ((n & 3) == 0 && n >= 24) eh_segment<4>(P, sg, want_h != 0, fsm);
    else if ((n & 1) == 0) eh_segment<2>(P, sg, want_h != 0, fsm);
    else eh_segment<1>(P, sg, want_h != 0, fsm);
  }
}

// ---------------------------------------------------------------- adjoint
// gD_i = -g_i x_i^T, gO_i = -(g_i x_{i+1}^T + x_i g_{i+1}^T), caller layout
// (row-major blocks).  One warp per block row: x_i, g_i, x_{i+1}, g_{i+1} are
// staged in shared memory, then the warp writes each n x n block as one flat
// range -- element f = a n + c, the lanes on consecutive pairs (f, f + 1)
// with 16-byte streaming stores when n is even and the block 16-byte
// aligned, single elements otherwise -- stepping (a, c) by carries instead of
// a division per element.  Bound by the (2N-1) n^2 doubles it writes.
constexpr int kAdjWarps = 8;

template <int W>  // elements per lane and store: 2 (double2) or 1
__device__ __forceinline__ void adj_block(double* dst, int n, const double* xa, const double* ga, const double* xb,
                                          const double* gb, bool off_diag, int lane) {
  const int nn = n * n, step = 32 * W;
  const int da = step / n, dc = step - da * n;
  int f = W * lane;
  int a = f / n, c = f - a * n;
  for (; f < nn; f += step) {
    double v[W];
#pragma unroll
    for (int w = 0; w < W; ++w)
      v[w] = off_diag ? -fma(ga[a], xb[c + w], xa[a] * gb[c + w]) : -ga[a] * xa[c + w];
    if constexpr (W == 2) __stcs(reinterpret_cast<double2*>(dst + f), make_double2(v[0], v[1]));
    else __stcs(dst + f, v[0]);
    a += da;
    c += dc;
    if (c >= n) {
      c -= n;
      ++a;
    }
  }
}

__global__ void __launch_bounds__(kAdjWarps * 32) k_adjoint(const __grid_constant__ AdjParams P) {
  __shared__ double stage[kAdjWarps][4][kMaxBlock];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long gr = (long long)blockIdx.x * kAdjWarps + warp;
  if (gr >= P.nrows) return;
  const RowRef rr = P.rows[gr];
  const InstDesc d = P.inst[rr.inst];
  const int n = d.n, i = rr.row;
  const bool has_next = i < d.N - 1;
  double* xs = stage[warp][0];  // x_i, g_i, x_{i+1}, g_{i+1}
  double* gs = stage[warp][1];
  double* xn = stage[warp][2];
  double* gn = stage[warp][3];
  const double* xi = P.x + d.vec + (long long)i * n;
  const double* gi = P.g + d.vec + (long long)i * n;
  for (int t = lane; t < n; t += 32) {
    xs[t] = xi[t];
    gs[t] = gi[t];
    if (has_next) {
      xn[t] = xi[n + t];
      gn[t] = gi[n + t];
    }
  }
  __syncwarp();
  double* gD = P.gD + P.d_off[rr.inst] + (long long)i * n * n;
  const bool pairs = (n % 2 == 0) && ((reinterpret_cast<uintptr_t>(gD) & 15) == 0);
  if (pairs) adj_block<2>(gD, n, xs, gs, nullptr, nullptr, false, lane);
  else adj_block<1>(gD, n, xs, gs, nullptr, nullptr, false, lane);
  if (has_next) {
    double* gO = P.gO + P.o_off[rr.inst] + (long long)i * n * n;
    if ((n % 2 == 0) && ((reinterpret_cast<uintptr_t>(gO) & 15) == 0)) adj_block<2>(gO, n, xs, gs, xn, gn, true, lane);
    else adj_block<1>(gO, n, xs, gs, xn, gn, true, lane);
  }
}

}  // namespace bt

// ---------------------------------------------------------------- host launchers
static cudaError_t launch_setup_opt(const bt::SetupParams* P, int mixed, int m, int maxn, cudaStream_t st) {
  const long long nb = P->nrows;
  if (nb == 0) return cudaSuccess;
  const dim3 grid((unsigned)nb);
  cudaError_t err;
  const int per_warp = 16 * maxn * maxn + 8 * bt::kMaxBlock;  // A | T | diagonal reciprocals
  int wpc = (200 * 1024) / per_warp;
  if (wpc > 8) wpc = 8;
  if (wpc < 1) wpc = 1;
  const dim3 fgrid((unsigned)((nb + wpc - 1) / wpc));
  const int sm_fac = wpc * per_warp;
  const int msz = mixed ? 4 : 8;
  const int sm_prod = 3 * maxn * maxn * msz;
  if (mixed && P->retry) {
    const int per_warp32 = (4 * maxn * (maxn + 1) + 15) / 16 * 16 + 64 * (int)sizeof(float);
    const int wpc32 = 4;  // register-resident factor: ~170 registers per thread
    const int sm32 = wpc32 * per_warp32;
    cudaFuncSetAttribute(bt::k_factor32, cudaFuncAttributeMaxDynamicSharedMemorySize, sm32);
    cudaFuncSetAttribute(bt::k_factor_retry, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_fac);
    cudaFuncSetAttribute(bt::k_E<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_prod);
    cudaFuncSetAttribute(bt::k_H<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_prod);
    if ((err = cudaMemsetAsync(P->retry, 0, sizeof(int), st)) != cudaSuccess) return err;
    if (P->cls_idx) {
      // one launch per block-size class: each kernel holds one variant and
      // takes its registers (n = 12 and 24 run at a higher occupancy than
      // next to the n = 36 variant)
      const auto launch_cls = [&](void (*kern)(bt::SetupParams, int, int, int), int c, int nbk) -> cudaError_t {
        const long long cnt = P->cls_hi[c] - P->cls_lo[c];
        if (cnt <= 0) return cudaSuccess;
        const int q = nbk > 0 ? nbk : maxn;
        const int pw = (4 * q * (q + 1) + 15) / 16 * 16 + 64 * (int)sizeof(float);
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, wpc32 * pw);
        if (e != cudaSuccess) return e;
        kern<<<(unsigned)((cnt + wpc32 - 1) / wpc32), 32 * wpc32, wpc32 * pw, st>>>(*P, wpc32, pw, c);
        return cudaGetLastError();
      };
      if ((err = launch_cls(bt::k_factor32_cls<12>, 0, 12)) != cudaSuccess) return err;
      if ((err = launch_cls(bt::k_factor32_cls<24>, 1, 24)) != cudaSuccess) return err;
      if ((err = launch_cls(bt::k_factor32_cls<36>, 2, 36)) != cudaSuccess) return err;
      if ((err = launch_cls(bt::k_factor32_cls<-1>, 3, 0)) != cudaSuccess) return err;
    } else {
      bt::k_factor32<<<(unsigned)((nb + wpc32 - 1) / wpc32), 32 * wpc32, sm32, st>>>(*P, wpc32, per_warp32);
      if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    const long long rgrid = std::min<long long>((nb + wpc - 1) / wpc, 304);
    bt::k_factor_retry<<<(unsigned)rgrid, 32 * wpc, sm_fac, st>>>(*P, wpc, per_warp);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    int maxbs = 0;  // largest float32 slot of any block size up to maxn
    for (int q = 1; q <= maxn; ++q) maxbs = std::max(maxbs, bt::slot32(q));
    const int sm_eh = bt::kEHSlots * maxbs * (int)sizeof(float);
    if (P->segs && P->nsegs > 0 && sm_eh <= 200 * 1024) {
      if (P->cls_idx) {  // the segments grouped by class: one launch per class
        const auto launch_cls = [&](void (*kern)(bt::SetupParams, int, int), int c, int nbk) -> cudaError_t {
          const long long cnt = P->seg_hi[c] - P->seg_lo[c];
          if (cnt <= 0) return cudaSuccess;
          const int smc = nbk > 0 ? bt::kEHSlots * bt::slot32(nbk) * (int)sizeof(float) : sm_eh;
          cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smc);
          if (e != cudaSuccess) return e;
          kern<<<(unsigned)cnt, 256, smc, st>>>(*P, m >= 2 ? 1 : 0, c);
          return cudaGetLastError();
        };
        if ((err = launch_cls(bt::k_EH_cls<2, 4>, 0, 12)) != cudaSuccess) return err;
        if ((err = launch_cls(bt::k_EH_cls<4, 4>, 1, 24)) != cudaSuccess) return err;
        if ((err = launch_cls(bt::k_EH_cls<4, 2>, 2, 36)) != cudaSuccess) return err;
        return launch_cls(bt::k_EH_cls<0, 2>, 3, 0);
      }
      cudaFuncSetAttribute(bt::k_EH, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_eh);
      bt::k_EH<<<(unsigned)P->nsegs, 256, sm_eh, st>>>(*P, m >= 2 ? 1 : 0);
      return cudaGetLastError();
    }
    bt::k_E<float><<<grid, 128, sm_prod, st>>>(*P);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if (m >= 2) bt::k_H<float><<<grid, 128, sm_prod, st>>>(*P);
  } else if (mixed) {
    cudaFuncSetAttribute(bt::k_factor<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_fac);
    cudaFuncSetAttribute(bt::k_E<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_prod);
    cudaFuncSetAttribute(bt::k_H<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_prod);
    bt::k_factor<float><<<fgrid, 32 * wpc, sm_fac, st>>>(*P, wpc, per_warp);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    bt::k_E<float><<<grid, 128, sm_prod, st>>>(*P);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if (m >= 2) bt::k_H<float><<<grid, 128, sm_prod, st>>>(*P);
  } else {
    cudaFuncSetAttribute(bt::k_factor<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_fac);
    cudaFuncSetAttribute(bt::k_E<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_prod);
    cudaFuncSetAttribute(bt::k_H<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_prod);
    bt::k_factor<double><<<fgrid, 32 * wpc, sm_fac, st>>>(*P, wpc, per_warp);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    bt::k_E<double><<<grid, 128, sm_prod, st>>>(*P);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if (m >= 2) bt::k_H<double><<<grid, 128, sm_prod, st>>>(*P);
  }
  return cudaGetLastError();
}

// Setup of the optimum (a = 1) blocks, then, for a general member of the
// family, the scaling by a and the +-1 blocks of H_ab (k_FK).
extern "C" cudaError_t bt_launch_setup(const bt::SetupParams* P, int mixed, int m, int maxn, cudaStream_t st) {
  cudaError_t err = launch_setup_opt(P, mixed, m, maxn, st);
  if (err != cudaSuccess || P->nrows == 0 || P->fam_a == 1.0) return err;
  const int sm_prod = 3 * maxn * maxn * (mixed ? 4 : 8);
  if (mixed) {
    cudaFuncSetAttribute(bt::k_FK<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_prod);
    bt::k_FK<float><<<(unsigned)P->nrows, 128, sm_prod, st>>>(*P);
  } else {
    cudaFuncSetAttribute(bt::k_FK<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_prod);
    bt::k_FK<double><<<(unsigned)P->nrows, 128, sm_prod, st>>>(*P);
  }
  return cudaGetLastError();
}

extern "C" cudaError_t bt_launch_adjoint(const bt::AdjParams* P, cudaStream_t st) {
  if (P->nrows == 0) return cudaSuccess;
  const long long grid = (P->nrows + bt::kAdjWarps - 1) / bt::kAdjWarps;
  bt::k_adjoint<<<(unsigned)grid, bt::kAdjWarps * 32, 0, st>>>(*P);
  return cudaGetLastError();
}
