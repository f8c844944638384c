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
#include "bt_common.cuh"

namespace bt {

// ---------------------------------------------------------------- K0+K1
// One warp per block row: load D_i (and O_i) once, write the library copies
// (column-major; float64 and, for mixed handles, float32), factor D_i by
// Cholesky in float64, invert the factor and form D_i^-1 = W^T W in MT.
// Warp-synchronous: no CTA barriers, so a CTA hosts several block rows.
template <typename MT>
__global__ void k_factor(const __grid_constant__ SetupParams P, int wpc, int warp_bytes) {
  extern __shared__ __align__(16) char smraw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long gr = (long long)blockIdx.x * wpc + warp;
  if (gr >= P.nrows) return;
  const RowRef rr = P.rows[gr];
  const InstDesc d = P.inst[rr.inst];
  const int n = d.n, i = rr.row, nn = n * n;
  double* A = reinterpret_cast<double*>(smraw + (size_t)warp * warp_bytes);  // 16 maxn^2 + 512 bytes per warp
  double* T = A + nn;
  const double* Du = P.D + P.d_off[rr.inst] + (long long)i * nn;
  const bool hasO = i < d.N - 1;
  for (int t = lane; t < nn; t += 32) A[t] = Du[t];
  if (hasO) {
    const double* Ou = P.O + P.o_off[rr.inst] + (long long)i * nn;
    for (int t = lane; t < nn; t += 32) T[t] = Ou[t];
  }
  __syncwarp();
  const float inv_n = 1.0f / (float)n;
  {
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
  // W = L^-1 (one column per lane, forward substitution in MT); the
  // reciprocals of the diagonal are formed once, into the warp's tail region.
  MT* W = reinterpret_cast<MT*>(T);
  // 1 / L[r][r] from the Cholesky; float32 copies sit behind W's float32 data
  MT* dv = (sizeof(MT) == 4) ? reinterpret_cast<MT*>(T) + nn : reinterpret_cast<MT*>(rinv_col);
  if (sizeof(MT) == 4)
    for (int r = lane; r < n; r += 32) dv[r] = (MT)rinv_col[r];
  __syncwarp();
  for (int c = lane; c < n; c += 32) {
    for (int r = 0; r < c; ++r) W[r * n + c] = MT(0);
    W[c * n + c] = dv[c];
    for (int r = c + 1; r < n; ++r) {
      MT acc = MT(0);
      for (int t = c; t < r; ++t) acc = fma((MT)A[r * n + t], W[t * n + c], acc);
      W[r * n + c] = -acc * dv[r];
    }
  }
  __syncwarp();
  MT* out = (sizeof(MT) == 8) ? reinterpret_cast<MT*>(P.Dinv64 + d.off64 + (long long)i * d.bs64)
                              : reinterpret_cast<MT*>(P.Dinv32 + d.off32 + (long long)i * d.bs32);
  for (int t = lane; t < nn; t += 32) {
    const int a = qdiv(t, inv_n), b = t - a * n;
    if (a < b) continue;
    MT acc = MT(0);
    for (int r = a; r < n; ++r) acc = fma(W[r * n + a], W[r * n + b], acc);
    out[(long long)b * n + a] = acc;
    out[(long long)a * n + b] = acc;
  }
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

// ---------------------------------------------------------------- adjoint
// gD_i = -g_i x_i^T, gO_i = -(g_i x_{i+1}^T + x_i g_{i+1}^T), caller layout.
__global__ void k_adjoint(const __grid_constant__ AdjParams P) {
  const long long gr = blockIdx.x;
  if (gr >= P.nrows) return;
  const RowRef rr = P.rows[gr];
  const InstDesc d = P.inst[rr.inst];
  const int n = d.n, i = rr.row;
  const double* x = P.x + d.vec;
  const double* g = P.g + d.vec;
  double* gD = P.gD + P.d_off[rr.inst] + (long long)i * n * n;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int a = t / n, c = t % n;
    gD[t] = -g[(long long)i * n + a] * x[(long long)i * n + c];
  }
  if (i < d.N - 1) {
    double* gO = P.gO + P.o_off[rr.inst] + (long long)i * n * n;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
      const int a = t / n, c = t % n;
      gO[t] = -(g[(long long)i * n + a] * x[(long long)(i + 1) * n + c] +
                x[(long long)i * n + a] * g[(long long)(i + 1) * n + c]);
    }
  }
}

}  // namespace bt

// ---------------------------------------------------------------- host launchers
extern "C" cudaError_t bt_launch_setup(const bt::SetupParams* P, int mixed, int m, int maxn, cudaStream_t st) {
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
  if (mixed) {
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

extern "C" cudaError_t bt_launch_adjoint(const bt::AdjParams* P, cudaStream_t st) {
  if (P->nrows == 0) return cudaSuccess;
  bt::k_adjoint<<<(unsigned)P->nrows, 128, 0, st>>>(*P);
  return cudaGetLastError();
}
