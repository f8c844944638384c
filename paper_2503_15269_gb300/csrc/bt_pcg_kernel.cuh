// Persistent PCG kernel for SPD block-tridiagonal systems with the optimal
// multi-splitting polynomial preconditioner (arXiv 2503.15269, a = 1, b = -1).
//
// One launch runs whole solves on the device.  Work units are instances;
// each is processed by a group of G CTAs that split its block rows into
// contiguous ranges (G = 1 in batched mode, where CTAs pull instances from a
// queue; G > 1 for one large instance, with a bounded global barrier).
//
// Every PCG iteration is a fixed sequence of sweeps over the block rows:
//   A   q = S p                  blocks D_i, O_i           (Eq. 1)
//   B1  y0 = G r                 blocks D_i^-1, E_i        (Sec. 4.1, Sec. 4.2)
//   B2  y_j = H y_{j-1}          blocks Hd_i, Hu_i, Hl_i   (Sec. 4.1, Sec. 4.2)
//  (A64 r64 = b - S x in float64 for the refinement of the mixed mode.)
// A general member of the family (a < 1, b = 1 - 2a) keeps the B1 sweep with
// E_i scaled by a at setup, and its H sweeps (B2G) stream five arrays: a Hd_i,
// a Hu_i, a Hl_i and the +-1 blocks F_i = -(1-a) D_i^-1 O_i and
// K_i = -(1-a) D_{i+1}^-1 O_i^T of H_ab = a H_J^2 + (1-a) H_J (Sec. 3.1).
// A sweep streams its blocks chunk by chunk through a ring of shared-memory
// stages filled by bulk asynchronous copies (TMA engine, mbarrier completion);
// the ring keeps prefetching along the predicted sweep sequence across sweep
// and iteration boundaries, and is drained only when the sequence breaks
// (convergence, end of a refinement step, next instance).
//
// Each row is processed in scatter form: row i computes its own direct terms
// (D_i p_i + O_i p_{i+1}; D_i^-1 r_i - E_i r_{i+1}; Hd_i y_i + Hu_i y_{i+2}) and
// pushes O_i^T p_i, -E_i^T r_i, Hl_i y_i to the row below, so a chunk needs no
// matrix block outside its own rows except at the start of a CTA's range
// (a halo of 1 or 2 push-only rows).  The vector updates of textbook PCG are
// fused into the staging of the sweep that first needs them.
#pragma once
#include "bt_common.cuh"

namespace bt {

// kKB2G: H_ab of a general member of the family (a < 1), five block arrays;
// kKJ: one application of H_J = -D^-1 (off-diagonal part of S), from D^-1 and O
// (the matrix-free H_opt = H_J^2 is two of them)
enum Kind : int { kKA = 0, kKB1 = 1, kKB2 = 2, kKA64 = 3, kKB2G = 4, kKJ = 5 };
enum StageMode : int { SV_P = 0, SV_VEC = 1, SV_R_UPD = 2, SV_R_FIRST = 3, SV_R_X0 = 4, SV_Y = 5 };
enum FinMode : int { FN_Q = 0, FN_OUT64 = 1, FN_R64 = 2, FN_Y0 = 3, FN_YJ = 4, FN_T = 5 };

// Per-kind chunk geometry.
struct Geo {
  int R;      // owned rows per chunk
  int halo;   // push-only rows before a CTA range start
  int k;      // push distance (1 for S and G, 2 for H)
  int narr;   // block arrays in the chunk
};

// `group`: the instance's rows are split over several CTAs, so the first chunk
// of a range may carry halo rows; a whole instance (batched mode) starts at
// row 0 and never does, and its stages need no slots for them.
__device__ __forceinline__ Geo geo_of(int kind, int stage_bytes, int bs_bytes, int n, bool group) {
  Geo g;
  const int slots = stage_bytes / bs_bytes;
  if (kind == kKB2) {
    g.R = (slots - (group ? 2 : 0)) / 3; g.halo = 2; g.k = 2; g.narr = 3;
  } else if (kind == kKB2G) {
    g.R = (slots - 4) / 5; g.halo = 2; g.k = 2; g.narr = 5;  // fixed stage layout (halo slots kept)
  } else {
    g.R = (slots - (group ? 1 : 0)) / 2; g.halo = 1; g.k = 1; g.narr = 2;
  }
  const int cap = kMaxChunkElems / n;
  if (g.R > cap) g.R = cap;
  if (g.R < 1) g.R = 1;
  return g;
}

// Smem carve-up (bytes).  Fixed part first, then the stages (128-aligned).
constexpr int kSmCtl = 0;                               // ints
constexpr int kSmRed = 128;                             // double [8 warps][4]
constexpr int kSmBc = kSmRed + (kThreads / 32) * 4 * 8;  // double bcast[8]
constexpr int kVsElems = kMaxChunkElems + 4 * kMaxBlock;
constexpr int kSmRing = kSmBc + 8 * 8;                  // T ring[2 buffers][2][64]
constexpr int kSmVs = kSmRing + 2 * 2 * kMaxBlock * 8;  // T vs[2 buffers][kVsElems]
constexpr int kSmParts = kSmVs + 2 * kVsElems * 8;      // T p1[512], p2[512], push[512+128]
constexpr int kSmFam = kSmParts + (3 * kMaxChunkElems + 2 * kMaxBlock) * 8;   // T part3[512], push1[512+128], ring1[2][64]
// the family region exists in the kernels of the general member only (GEN)
template <bool GEN>
constexpr int kSmFull = GEN ? kSmFam + (2 * kMaxChunkElems + 4 * kMaxBlock) * 8 : kSmFam;  // uint64 full[kMaxStages]
constexpr int kVecSlots = 4;  // vector ring slots at most (the general member's kernels use 3)
template <bool GEN>
constexpr int kSmVbar = kSmFull<GEN> + kMaxStages * 8;         // uint64 vbar[kVecSlots]
template <bool GEN>
constexpr int kSmVring = ((kSmVbar<GEN> + kVecSlots * 8 + 127) / 128) * 128;  // vector ring, then the stages

// fixed part; the host adds (4, or 3 for the general member) * vec_slot_bytes
// + stages * stage_bytes
template <bool GEN>
__host__ __device__ constexpr int smem_fixed_bytes() { return kSmVring<GEN>; }

template <typename T>
__device__ __forceinline__ T dot_col(const T* __restrict__ M, int n, int a, const T* __restrict__ v) {
  // (M v)[a] with M column-major: element (a, c) at c*n + a.
  T acc0 = T(0), acc1 = T(0);
  int c = 0;
  for (; c + 1 < n; c += 2) {
    acc0 = fma(M[c * n + a], v[c], acc0);
    acc1 = fma(M[(c + 1) * n + a], v[c + 1], acc1);
  }
  if (c < n) acc0 = fma(M[c * n + a], v[c], acc0);
  return acc0 + acc1;
}

template <typename T>
__device__ __forceinline__ T dot_tr(const T* __restrict__ M, int n, int a, const T* __restrict__ v) {
  // (M^T v)[a] = sum_c M(c, a) v[c]; column a is contiguous.
  const T* col = M + a * n;
  T acc0 = T(0), acc1 = T(0);
  int c = 0;
  for (; c + 1 < n; c += 2) {
    acc0 = fma(col[c], v[c], acc0);
    acc1 = fma(col[c + 1], v[c + 1], acc1);
  }
  if (c < n) acc0 = fma(col[c], v[c], acc0);
  return acc0 + acc1;
}

// Description of one sweep (uniform across the CTA).
template <typename T>
struct Sweep {
  int kind;
  int stg, fin;
  // staging inputs
  const T* z; const T* p_old; T* p_cur;             // SV_P
  const double* src64; double scale;                // SV_VEC / SV_R_FIRST / SV_R_X0
  const T* r_old; const T* q; T* r_cur; T* x; const T* p_in;  // SV_R_UPD
  bool write_r, write_x, zero_x;
  const T* yprev;                                   // SV_Y
  T alpha, beta;                                    // PCG scalars (cast)
  bool first;                                       // SV_P with beta = 0
  // finalize outputs
  T* qout; double* out64; const double* bsub;       // FN_Q / FN_OUT64 / FN_R64
  double* r64;
  T* y0; T* ynext; T* zv; const T* rcur_for_dot;    // FN_Y0 / FN_YJ
  int j, m; T alpha_j; bool last, out_to_user, m1;
  T sgn;
};


template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// Two outputs (a, a+1) of M v, M column-major NB x NB, a even.
template <int NB, typename T>
__device__ __forceinline__ void dcol2(const T* __restrict__ M, int a, const T* __restrict__ v, T& o0, T& o1) {
  using V = typename Vec2<T>::type;
  T a0 = T(0), a1 = T(0), b0 = T(0), b1 = T(0);
  if constexpr (sizeof(T) == 4 && NB % 4 == 0) {  // v four words per load
#pragma unroll
    for (int c = 0; c < NB; c += 4) {
      const float4 vv = *reinterpret_cast<const float4*>(v + c);
      const V m0 = *reinterpret_cast<const V*>(M + c * NB + a);
      const V m1 = *reinterpret_cast<const V*>(M + (c + 1) * NB + a);
      const V m2 = *reinterpret_cast<const V*>(M + (c + 2) * NB + a);
      const V m3 = *reinterpret_cast<const V*>(M + (c + 3) * NB + a);
      a0 = fma(m0.x, vv.x, a0);
      a1 = fma(m0.y, vv.x, a1);
      b0 = fma(m1.x, vv.y, b0);
      b1 = fma(m1.y, vv.y, b1);
      a0 = fma(m2.x, vv.z, a0);
      a1 = fma(m2.y, vv.z, a1);
      b0 = fma(m3.x, vv.w, b0);
      b1 = fma(m3.y, vv.w, b1);
    }
  } else {
#pragma unroll
    for (int c = 0; c < NB; c += 2) {
      const V m0 = *reinterpret_cast<const V*>(M + c * NB + a);
      const V m1 = *reinterpret_cast<const V*>(M + (c + 1) * NB + a);
      const V vv = *reinterpret_cast<const V*>(v + c);
      a0 = fma(m0.x, vv.x, a0);
      a1 = fma(m0.y, vv.x, a1);
      b0 = fma(m1.x, vv.y, b0);
      b1 = fma(m1.y, vv.y, b1);
    }
  }
  o0 = a0 + b0;
  o1 = a1 + b1;
}

// One output of M^T v: column a of M (contiguous) dotted with v.  The walk
// along the column starts at an offset chosen per lane so that the 8 lanes
// of a 128-bit shared-memory phase (consecutive a) fall in distinct bank
// groups: word n*a + 4*q sits in bank group (n/4*a + q) mod 8, already
// distinct for n = 4 mod 8; n = 24 adds (a >> 2) & 1 and n = 48 (a >> 1) & 3.
template <int NB>
__device__ __forceinline__ int tr_rot(int a) {
  if constexpr (NB % 8 == 4) return 0;
  else if constexpr (NB % 32 == 24 || NB % 32 == 8) return (a >> 2) & 1;
  else return (a >> 1) & 3;
}

template <int NB, typename T>
__device__ __forceinline__ T dtr1(const T* __restrict__ M, int a, const T* __restrict__ v, int /*unused*/) {
  constexpr int Q = NB / 4;
  const T* col = M + a * NB;
  const int rot = tr_rot<NB>(a) % Q;
  T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    int qq = q + rot;
    if (qq >= Q) qq -= Q;
    if constexpr (sizeof(T) == 4) {
      const float4 m = *reinterpret_cast<const float4*>(col + 4 * qq);
      const float4 w = *reinterpret_cast<const float4*>(v + 4 * qq);
      s0 = fma(m.x, w.x, s0);
      s1 = fma(m.y, w.y, s1);
      s2 = fma(m.z, w.z, s2);
      s3 = fma(m.w, w.w, s3);
    } else {
      using V = typename Vec2<T>::type;
      const V m0 = *reinterpret_cast<const V*>(col + 4 * qq);
      const V m1 = *reinterpret_cast<const V*>(col + 4 * qq + 2);
      const V v0 = *reinterpret_cast<const V*>(v + 4 * qq);
      const V v1 = *reinterpret_cast<const V*>(v + 4 * qq + 2);
      s0 = fma(m0.x, v0.x, s0);
      s1 = fma(m0.y, v0.y, s1);
      s2 = fma(m1.x, v1.x, s2);
      s3 = fma(m1.y, v1.y, s3);
    }
  }
  return (s0 + s1) + (s2 + s3);
}

// Four outputs (a .. a+3) of M v, M float32 column-major NB x NB, a % 4 == 0:
// one 128-bit load per column step of M and one per four entries of v.
template <int NB>
__device__ __forceinline__ float4 dcol4(const float* __restrict__ M, int a, const float* __restrict__ v) {
  float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0;
#pragma unroll
  for (int c = 0; c < NB; c += 4) {
    const float4 vv = *reinterpret_cast<const float4*>(v + c);
    const float4 m0 = *reinterpret_cast<const float4*>(M + c * NB + a);
    const float4 m1 = *reinterpret_cast<const float4*>(M + (c + 1) * NB + a);
    const float4 m2 = *reinterpret_cast<const float4*>(M + (c + 2) * NB + a);
    const float4 m3 = *reinterpret_cast<const float4*>(M + (c + 3) * NB + a);
    s0 = make_float4(fmaf(m0.x, vv.x, s0.x), fmaf(m0.y, vv.x, s0.y), fmaf(m0.z, vv.x, s0.z), fmaf(m0.w, vv.x, s0.w));
    s1 = make_float4(fmaf(m1.x, vv.y, s1.x), fmaf(m1.y, vv.y, s1.y), fmaf(m1.z, vv.y, s1.z), fmaf(m1.w, vv.y, s1.w));
    s0 = make_float4(fmaf(m2.x, vv.z, s0.x), fmaf(m2.y, vv.z, s0.y), fmaf(m2.z, vv.z, s0.z), fmaf(m2.w, vv.z, s0.w));
    s1 = make_float4(fmaf(m3.x, vv.w, s1.x), fmaf(m3.y, vv.w, s1.y), fmaf(m3.z, vv.w, s1.z), fmaf(m3.w, vv.w, s1.w));
  }
  return make_float4(s0.x + s1.x, s0.y + s1.y, s0.z + s1.z, s0.w + s1.w);
}

// Start offset of the column walk of dtr2 for the column pair p = a / 2:
// pair p reads words 2 p NB + 4 q (and NB more), bank group (p NB / 2 + q)
// mod 8, so the 8 lanes of a 128-bit phase need distinct (p NB / 2 + rot)
// mod 8: NB = 4 mod 8 repeats every 4 pairs, NB = 8 mod 16 every 2, and
// NB = 0 mod 16 at once.
template <int NB>
__device__ __forceinline__ int tr2_rot(int p) {
  if constexpr (NB % 8 == 4) return (p >> 2) & 1;
  else if constexpr (NB % 16 == 8) return (p >> 1) & 3;
  else return p & 7;
}

// Two outputs (a, a+1) of M^T v, M float32 column-major NB x NB, a even:
// columns a and a+1 of M (contiguous) dotted with v.
template <int NB>
__device__ __forceinline__ float2 dtr2(const float* __restrict__ M, int a, const float* __restrict__ v) {
  constexpr int Q = NB / 4;
  const float* c0 = M + a * NB;
  const float* c1 = c0 + NB;
  const int rot = tr2_rot<NB>(a >> 1) % Q;
  float x0 = 0.f, x1 = 0.f, y0 = 0.f, y1 = 0.f;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    int qq = q + rot;
    if (qq >= Q) qq -= Q;
    const float4 w = *reinterpret_cast<const float4*>(v + 4 * qq);
    const float4 m0 = *reinterpret_cast<const float4*>(c0 + 4 * qq);
    const float4 m1 = *reinterpret_cast<const float4*>(c1 + 4 * qq);
    x0 = fmaf(m0.x, w.x, x0);
    x1 = fmaf(m0.y, w.y, x1);
    y0 = fmaf(m1.x, w.x, y0);
    y1 = fmaf(m1.y, w.y, y1);
    x0 = fmaf(m0.z, w.z, x0);
    x1 = fmaf(m0.w, w.w, x1);
    y0 = fmaf(m1.z, w.z, y0);
    y1 = fmaf(m1.w, w.w, y1);
  }
  return make_float2(x0 + x1, y0 + y1);
}

// All block-vector products of one chunk: part1 = M1 v_i, part2 = M2 v_{i+k},
// push = (M2^T v_i) for S and G, (Hl_i v_i) for H.  For H_ab (kKB2G) also
// part3 = F_i v_{i+1} and push1 = K_i v_i (to row i+1).  NB = 0: runtime n.
template <int KIND, int NB, typename T>
__device__ __forceinline__ void chunk_products(const T* __restrict__ stg, int R, int bse, int n_rt, int N, int nr,
                                               int h, int r0, int base, const T* __restrict__ vs, T* part1, T* part2,
                                               T* push, T* part3, T* push1) {
  constexpr int k = (KIND == kKB2 || KIND == kKB2G) ? 2 : 1;
  const int tid = threadIdx.x;
  const T* a0 = stg;
  const T* a1 = stg + (size_t)R * bse;
  const T* a2 = stg + (size_t)2 * R * bse;
  if constexpr (KIND == kKJ) {
    // stage: D^-1 [R] | O [R+1]; first phase of H_J v: part2 = O_i v_{i+1},
    // push = O_i^T v_i (to row i+1); D^-1 is applied in a second phase
    if constexpr (NB > 0) {
      constexpr int n = NB;
      constexpr int hp = NB / 2;
      const int nd2 = nr * hp;
      const int np = (nr + h) * n;
      for (int t = tid; t < nd2 + np; t += kThreads) {
        if (t < nd2) {
          const int jj = t / hp, a = 2 * (t - jj * hp);
          if (r0 + jj + 1 < N) {
            dcol2<NB>(a1 + (size_t)(jj + h) * bse, a, vs + (r0 + jj + 1 - base) * n, part2[jj * n + a],
                      part2[jj * n + a + 1]);
          } else {
            part2[jj * n + a] = T(0);
            part2[jj * n + a + 1] = T(0);
          }
        } else {
          const int t3 = t - nd2;
          const int jj = t3 / n, a = t3 - jj * n;
          push[jj * n + a] = dtr1<NB>(a1 + (size_t)jj * bse, a, vs + jj * n, 0);
        }
      }
    } else {
      const int n = n_rt;
      const int nd = nr * n, np = (nr + h) * n;
      for (int t = tid; t < nd + np; t += kThreads) {
        if (t < nd) {
          const int jj = t / n, a = t - jj * n;
          T val = T(0);
          if (r0 + jj + 1 < N) val = dot_col(a1 + (size_t)(jj + h) * bse, n, a, vs + (r0 + jj + 1 - base) * n);
          part2[t] = val;
        } else {
          const int t3 = t - nd;
          const int jj = t3 / n, a = t3 - jj * n;
          push[t3] = dot_tr(a1 + (size_t)jj * bse, n, a, vs + jj * n);
        }
      }
    }
    return;
  }
  if constexpr (KIND == kKB2G) {
    // stage: Hd [R] | Hu [R] | Hl [R+2] | F [R] | K [R+2]; every product is a
    // direct (column-major) one, the two lower bands are pushed forward
    const T* a3 = stg + (size_t)(3 * R + 2) * bse;
    const T* a4 = stg + (size_t)(4 * R + 2) * bse;
    if constexpr (NB > 0) {
      constexpr int n = NB;
      constexpr int hp = NB / 2;
      const int nd2 = nr * hp, np = (nr + h) * hp;
      const int ntask = 3 * nd2 + 2 * np;
      for (int t = tid; t < ntask; t += kThreads) {
        if (t < nd2) {
          const int jj = t / hp, a = 2 * (t - jj * hp);
          dcol2<NB>(a0 + (size_t)jj * bse, a, vs + (r0 + jj - base) * n, part1[jj * n + a], part1[jj * n + a + 1]);
        } else if (t < 3 * nd2) {
          const bool up2 = t < 2 * nd2;
          const int t2 = t - (up2 ? nd2 : 2 * nd2);
          const int jj = t2 / hp, a = 2 * (t2 - jj * hp);
          const int d = up2 ? 2 : 1;
          T* out = (up2 ? part2 : part3) + jj * n + a;
          if (r0 + jj + d < N) {
            dcol2<NB>((up2 ? a1 : a3) + (size_t)jj * bse, a, vs + (r0 + jj + d - base) * n, out[0], out[1]);
          } else {
            out[0] = T(0);
            out[1] = T(0);
          }
        } else {
          const bool p2 = t < 3 * nd2 + np;
          const int t3 = t - (p2 ? 3 * nd2 : 3 * nd2 + np);
          const int jj = t3 / hp, a = 2 * (t3 - jj * hp);
          T* out = (p2 ? push : push1) + jj * n + a;
          dcol2<NB>((p2 ? a2 : a4) + (size_t)jj * bse, a, vs + jj * n, out[0], out[1]);
        }
      }
    } else {
      const int n = n_rt;
      const int nd = nr * n, np = (nr + h) * n;
      const int ntask = 3 * nd + 2 * np;
      for (int t = tid; t < ntask; t += kThreads) {
        if (t < nd) {
          const int jj = t / n, a = t - jj * n;
          part1[t] = dot_col(a0 + (size_t)jj * bse, n, a, vs + (r0 + jj - base) * n);
        } else if (t < 3 * nd) {
          const bool up2 = t < 2 * nd;
          const int t2 = t - (up2 ? nd : 2 * nd);
          const int jj = t2 / n, a = t2 - jj * n;
          const int d = up2 ? 2 : 1;
          T val = T(0);
          if (r0 + jj + d < N) val = dot_col((up2 ? a1 : a3) + (size_t)jj * bse, n, a, vs + (r0 + jj + d - base) * n);
          (up2 ? part2 : part3)[t2] = val;
        } else {
          const bool p2 = t < 3 * nd + np;
          const int t3 = t - (p2 ? 3 * nd : 3 * nd + np);
          const int jj = t3 / n, a = t3 - jj * n;
          (p2 ? push : push1)[t3] = dot_col((p2 ? a2 : a4) + (size_t)jj * bse, n, a, vs + jj * n);
        }
      }
    }
    return;
  }
  if constexpr (NB > 0 && NB % 4 == 0 && NB <= 24 && sizeof(T) == 4) {
    // float32 blocks up to n = 24: four outputs of a direct product per
    // task, two of a transposed one (the push of S and G) -- half the tasks
    // of the two-output form, whose per-task overhead weighs most on small
    // blocks (n = 36 measured no faster this way)
    constexpr int n = NB;
    constexpr int q4 = NB / 4;
    constexpr int hp = NB / 2;
    const int nd4 = nr * q4;
    const int np = (KIND == kKB2) ? (nr + h) * q4 : (nr + h) * hp;
    const int ntask = 2 * nd4 + np;
    for (int t = tid; t < ntask; t += kThreads) {
      if (t < nd4) {
        const int jj = t / q4, a = 4 * (t - jj * q4);
        *reinterpret_cast<float4*>(part1 + jj * n + a) = dcol4<NB>(a0 + (size_t)jj * bse, a, vs + (r0 + jj - base) * n);
      } else if (t < 2 * nd4) {
        const int t2 = t - nd4;
        const int jj = t2 / q4, a = 4 * (t2 - jj * q4);
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r0 + jj + k < N) {
          const T* M2 = (KIND == kKB2) ? a1 + (size_t)jj * bse : a1 + (size_t)(jj + h) * bse;
          o = dcol4<NB>(M2, a, vs + (r0 + jj + k - base) * n);
        }
        *reinterpret_cast<float4*>(part2 + jj * n + a) = o;
      } else {
        const int t3 = t - 2 * nd4;
        if constexpr (KIND == kKB2) {
          const int jj = t3 / q4, a = 4 * (t3 - jj * q4);
          *reinterpret_cast<float4*>(push + jj * n + a) = dcol4<NB>(a2 + (size_t)jj * bse, a, vs + jj * n);
        } else {
          const int jj = t3 / hp, a = 2 * (t3 - jj * hp);
          *reinterpret_cast<float2*>(push + jj * n + a) = dtr2<NB>(a1 + (size_t)jj * bse, a, vs + jj * n);
        }
      }
    }
  } else if constexpr (NB > 0) {
    constexpr int n = NB;
    constexpr int hp = NB / 2;
    const int nd2 = nr * hp;                          // pairs of direct outputs
    const int np = (KIND == kKB2) ? (nr + h) * hp : (nr + h) * n;
    const int ntask = 2 * nd2 + np;
    for (int t = tid; t < ntask; t += kThreads) {
      if (t < nd2) {
        const int jj = t / hp, a = 2 * (t - jj * hp);
        dcol2<NB>(a0 + (size_t)jj * bse, a, vs + (r0 + jj - base) * n, part1[jj * n + a], part1[jj * n + a + 1]);
      } else if (t < 2 * nd2) {
        const int t2 = t - nd2;
        const int jj = t2 / hp, a = 2 * (t2 - jj * hp);
        if (r0 + jj + k < N) {
          const T* M2 = (KIND == kKB2) ? a1 + (size_t)jj * bse : a1 + (size_t)(jj + h) * bse;
          dcol2<NB>(M2, a, vs + (r0 + jj + k - base) * n, part2[jj * n + a], part2[jj * n + a + 1]);
        } else {
          part2[jj * n + a] = T(0);
          part2[jj * n + a + 1] = T(0);
        }
      } else {
        const int t3 = t - 2 * nd2;
        if constexpr (KIND == kKB2) {
          const int jj = t3 / hp, a = 2 * (t3 - jj * hp);
          dcol2<NB>(a2 + (size_t)jj * bse, a, vs + jj * n, push[jj * n + a], push[jj * n + a + 1]);
        } else {
          const int jj = t3 / n, a = t3 - jj * n;
          push[jj * n + a] = dtr1<NB>(a1 + (size_t)jj * bse, a, vs + jj * n, 0);
        }
      }
    }
  } else {
    // runtime block size (any n)
    const int n = n_rt;
    const int nd = nr * n;
    const int ntask = 2 * nd + (nr + h) * n;
    for (int t = tid; t < ntask; t += kThreads) {
      if (t < nd) {
        const int jj = t / n, a = t - jj * n;
        part1[t] = dot_col(a0 + (size_t)jj * bse, n, a, vs + (r0 + jj - base) * n);
      } else if (t < 2 * nd) {
        const int t2 = t - nd;
        const int jj = t2 / n, a = t2 - jj * n;
        T val = T(0);
        if (r0 + jj + k < N) {
          const T* M2 = (KIND == kKB2) ? a1 + (size_t)jj * bse : a1 + (size_t)(jj + h) * bse;
          val = dot_col(M2, n, a, vs + (r0 + jj + k - base) * n);
        }
        part2[t2] = val;
      } else {
        const int t3 = t - 2 * nd;
        const int jj = t3 / n, a = t3 - jj * n;
        if (KIND == kKB2) push[t3] = dot_col(a2 + (size_t)jj * bse, n, a, vs + jj * n);
        else push[t3] = dot_tr(a1 + (size_t)jj * bse, n, a, vs + jj * n);
      }
    }
  }
}

// Second phase of a kKJ chunk: out_i = D^-1_i s_i over the owned rows
// (D^-1 in the first R slots of the stage, s in shared memory).
template <int NB, typename T>
__device__ __forceinline__ void chunk_dinv(const T* __restrict__ a0, int bse, int n_rt, int nr,
                                           const T* __restrict__ s, T* out) {
  const int tid = threadIdx.x;
  if constexpr (NB > 0) {
    constexpr int hp = NB / 2;
    for (int t = tid; t < nr * hp; t += kThreads) {
      const int jj = t / hp, a = 2 * (t - jj * hp);
      dcol2<NB>(a0 + (size_t)jj * bse, a, s + jj * NB, out[jj * NB + a], out[jj * NB + a + 1]);
    }
  } else {
    const int n = n_rt;
    for (int t = tid; t < nr * n; t += kThreads) {
      const int jj = t / n, a = t - jj * n;
      out[t] = dot_col(a0 + (size_t)jj * bse, n, a, s + jj * n);
    }
  }
}

__device__ __forceinline__ float4 ld4f(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4f(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float4 fma4(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
// Dot-product partials.  Float64 issues at 1/64 of the float32 rate on this
// part, so the float32 sweeps keep float64 off the per-chunk path: each
// thread sums its float32 products (4-term dots) with a compensated float32
// sum (TwoSum: the rounding error of every addition is carried in c, so the
// partial is accurate to a few float32 ulps whatever the number of terms)
// and widens it once per sweep.  The float64 sweeps sum in float64.
__device__ __forceinline__ float dot4f(float4 a, float4 b) {
  return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x)));
}
// VAR: 0 = the optimum with stored H_opt; 1 = a general member of the family
// (a < 1, H sweeps of kind kKB2G); 2 = the optimum with the matrix-free
// H_opt = H_J^2 (two kKJ sweeps per application, no H blocks stored).  Each
// variant is its own kernel: the optimum's carries none of the others' code
// or shared memory.
template <typename MT, int VAR>
struct Solver {
  static constexpr bool GEN = (VAR == 1);
  static constexpr bool MF = (VAR == 2);
  static constexpr int kHK = GEN ? kKB2G : (MF ? kKJ : kKB2);  // kind of the H sweeps
  static constexpr int kHPS = MF ? 2 : 1;                      // sweeps per H application
  // vector ring slots: 4 (the pipelined sweeps keep a chunk's slot one phase
  // longer); 3 for the general member, whose extra shared memory leaves no
  // room for a fourth
  static constexpr int kVS = GEN ? 3 : kVecSlots;
  const KParams& P;
  char* sm;
  int tid;
  // group / instance
  int g, G;
  int N, n, s, e;
  long long vec;
  long long deadline;
  int bar_count;
  bool fail;
  int status;
  // pipeline
  int S, SB;
  uint64_t* full;
  char* stages;
  unsigned issued, consumed;
  // vector ring (bulk copies of the vector rows of a chunk, within a sweep)
  uint64_t* vbar;
  char* vring;
  int VSB;
  unsigned vissued, vcons;
  int pat_len, pat_first, p_slot, p_chunk;  // predicted sweep sequence (see kind_at)
  int ncA, ncB1, ncB2, ncA64;                // chunks per sweep kind for this instance
  const double* mats64[7];
  const MT* mats[GEN ? 9 : 7];
  int bs, bs64;

  __device__ Solver(const KParams& P_, char* sm_) : P(P_), sm(sm_) {
    tid = threadIdx.x;
    S = P.stages;
    SB = P.stage_bytes;
    full = reinterpret_cast<uint64_t*>(sm + kSmFull<GEN>);
    vbar = reinterpret_cast<uint64_t*>(sm + kSmVbar<GEN>);
    vring = sm + kSmVring<GEN>;
    VSB = P.vec_slot_bytes;
    stages = vring + (size_t)kVS * VSB;
    issued = consumed = 0;
    vissued = vcons = 0;
    bar_count = 0;
  }

  // ---- chunk geometry ----------------------------------------------------
  __device__ int bsb_of(int kind) const { return kind == kKA64 ? bs64 * 8 : bs * (int)sizeof(MT); }
  __device__ Geo geo(int kind) const { return geo_of(kind, SB, bsb_of(kind), n, G > 1); }
  __device__ int nchunks(int kind) const {
    Geo gg = geo(kind);
    return (e - s + gg.R - 1) / gg.R;
  }

  // ---- producer ------------------------------------------------------------
  // The pipeline state lives in a Producer value: sweeps copy it into
  // registers on entry and back on exit, so the per-chunk bookkeeping never
  // touches local memory.  The predicted sweep sequence is either a single
  // kind repeated (len 1) or the PCG iteration pattern A, B1, B2 x (m-1).
  struct Producer {
    int s, e, n, S, SB, bs, bs64;
    char* stages;
    uint64_t* full;
    const char *m0, *m1, *m2, *m3, *m4, *m5, *m6;  // D, O, D^-1, E, Hd, Hu, Hl (working precision)
    const char *m7, *m8;                            // F, K of H_ab (general member only)
    const char *d64, *o64;                          // float64 D, O
    int pat_len, pat_first, p_slot, p_chunk;
    int ncA, ncB1, ncB2, ncA64;
    int RA, RB1, RB2, RA64;
    unsigned issued;

    __device__ __forceinline__ int kind_at(int slot) const {
      return pat_len == 1 ? pat_first : (slot == 0 ? kKA : (slot == 1 ? kKB1 : kHK));
    }
    // the H counts and rows are those of the handle's H kind (kKB2 or kKB2G)
    __device__ __forceinline__ int nch(int kind) const {
      return kind == kKA ? ncA : (kind == kKB1 ? ncB1 : (kind == kKA64 ? ncA64 : ncB2));
    }
    __device__ __forceinline__ int rows(int kind) const {
      return kind == kKA ? RA : (kind == kKB1 ? RB1 : (kind == kKA64 ? RA64 : RB2));
    }
    // thread 0 issues the bulk copies of chunk c of `kind`; every thread
    // advances the cursor identically.
    __device__ __forceinline__ void step(bool leader) {
      const int kind = kind_at(p_slot);
      if (leader) {
        const int R = rows(kind);
        const int c = p_chunk;
        const int r0 = s + c * R;
        const int r1 = min(e, r0 + R);
        const int halo = (kind == kKB2 || (GEN && kind == kKB2G)) ? 2 : 1;
        const int h = (c == 0) ? min(halo, s) : 0;
        const int bse = (kind == kKA64) ? bs64 : bs;
        const int esz = (kind == kKA64) ? 8 : (int)sizeof(MT);
        const int bsb = bse * esz;
        const int st = issued % S;
        char* dst = stages + (size_t)st * SB;
        uint64_t* bar = &full[st];
        const int nr = r1 - r0;
        const bool hkind = (kind == kKB2 || (GEN && kind == kKB2G));
        const unsigned total =
            (unsigned)((GEN && kind == kKB2G) ? 5 * nr + 2 * h : ((kind == kKB2 ? 3 * nr : 2 * nr) + h)) * bsb;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar, total);
        const bool kj = MF && kind == kKJ;
        const char* A0 = kind == kKA ? m0 : ((kind == kKB1 || kj) ? m2 : (hkind ? m4 : d64));
        const char* A1 = kind == kKA ? m1 : (kind == kKB1 ? m3 : (hkind ? m5 : (kj ? m1 : o64)));
        bulk_g2s(dst, A0 + (size_t)r0 * bsb, nr * bsb, bar);
        if (hkind) {
          bulk_g2s(dst + (size_t)R * bsb, A1 + (size_t)r0 * bsb, nr * bsb, bar);
          bulk_g2s(dst + (size_t)2 * R * bsb, m6 + (size_t)(r0 - h) * bsb, (nr + h) * bsb, bar);
          if constexpr (GEN) {
            if (kind == kKB2G) {
              bulk_g2s(dst + (size_t)(3 * R + 2) * bsb, m7 + (size_t)r0 * bsb, nr * bsb, bar);
              bulk_g2s(dst + (size_t)(4 * R + 2) * bsb, m8 + (size_t)(r0 - h) * bsb, (nr + h) * bsb, bar);
            }
          }
        } else {
          bulk_g2s(dst + (size_t)R * bsb, A1 + (size_t)(r0 - h) * bsb, (nr + h) * bsb, bar);
        }
      }
      ++issued;
      if (++p_chunk >= nch(kind)) {
        p_chunk = 0;
        p_slot = (p_slot + 1 == pat_len) ? 0 : p_slot + 1;
      }
    }
  };

  __device__ __forceinline__ Producer producer() const {
    Producer q;
    q.s = s; q.e = e; q.n = n; q.S = S; q.SB = SB; q.bs = bs; q.bs64 = bs64;
    q.stages = stages; q.full = full;
    q.m0 = (const char*)mats[0]; q.m1 = (const char*)mats[1]; q.m2 = (const char*)mats[2];
    q.m3 = (const char*)mats[3]; q.m4 = (const char*)mats[4]; q.m5 = (const char*)mats[5];
    q.m6 = (const char*)mats[6];
    if constexpr (GEN) { q.m7 = (const char*)mats[7]; q.m8 = (const char*)mats[8]; }
    q.d64 = (const char*)mats64[0]; q.o64 = (const char*)mats64[1];
    q.pat_len = pat_len; q.pat_first = pat_first; q.p_slot = p_slot; q.p_chunk = p_chunk;
    q.ncA = ncA; q.ncB1 = ncB1; q.ncB2 = ncB2; q.ncA64 = ncA64;
    q.RA = geo(kKA).R; q.RB1 = geo(kKB1).R; q.RB2 = geo(kHK).R; q.RA64 = geo(kKA64).R;
    q.issued = issued;
    return q;
  }
  __device__ __forceinline__ void store_producer(const Producer& q) {
    p_slot = q.p_slot;
    p_chunk = q.p_chunk;
    issued = q.issued;
  }

  // chunk counts of the current instance (call after s, e, n, bs are set)
  __device__ void set_chunk_counts() {
    ncA = nchunks(kKA);
    ncB1 = nchunks(kKB1);
    ncB2 = nchunks(kHK);
    ncA64 = nchunks(kKA64);
  }

  // Drain every chunk in flight (bounded) so that the ring is idle.
  __device__ void flush() {
    bool ok = true;
    while (vcons < vissued) {
      const int st = vcons % kVS;
      const unsigned par = (vcons / kVS) & 1u;
      if (ok && !mbar_wait(&vbar[st], par, deadline + (1ll << 31))) ok = false;
      ++vcons;
    }
    while (consumed < issued) {
      const int st = consumed % S;
      const unsigned par = (consumed / S) & 1u;
      if (ok && !mbar_wait(&full[st], par, deadline + (1ll << 31))) ok = false;
      ++consumed;
    }
    __syncthreads();
    if (!ok) fail = true;
  }

  // Start a new predicted sweep sequence: either `first` repeated (len 1) or
  // the iteration pattern (len m + 1), from `start_slot`; prefill the ring.
  __device__ void restart(int first, int len, int start_slot) {
    flush();
    pat_len = len;
    pat_first = first;
    p_slot = start_slot;
    p_chunk = 0;
    Producer q = producer();
    for (int i = 0; i < S; ++i) q.step(tid == kLeaderTid);
    store_producer(q);
  }

  // ---- reductions & group barrier ----------------------------------------
  // Reduce 4 per-thread partials over the CTA, then over the group (fixed
  // order, so results are bitwise reproducible).  v[3] carries a timeout flag.
  __device__ void group_reduce(double v[4]) {
    if (fail) return;
    // vector rows written so far are read by bulk copies after this barrier
    fence_proxy_async_global();
    double* bc = reinterpret_cast<double*>(sm + kSmBc);
    int* ctl = reinterpret_cast<int*>(sm + kSmCtl);
    // Sum of the 3 x kThreads partials as a fixed tree spread over the
    // warps: every float64 add holds an SM sub-partition's float64 pipe for
    // ~64 cycles, so the adds go where the pipes are idle (four partials
    // per thread on 3 x 64 threads, then one warp per quantity) instead of
    // a shuffle tree in every warp and a serial sum on one thread.  The
    // vector staging buffers are free between sweeps.
    static_assert(kThreads % 64 == 0 && kThreads >= 192, "three quantities of 64 threads");
    double* tr = reinterpret_cast<double*>(sm + kSmVs);  // [3][kThreads] then [3][64]
    static_assert((3 * kThreads + 3 * 64) * 8 <= 2 * kVsElems * 8, "reduction scratch fits the staging buffers");
#pragma unroll
    for (int i = 0; i < 3; ++i) tr[i * kThreads + tid] = v[i];  // v[3] is set below (timeout flag)
    __syncthreads();
    if (tid < 3 * 64) {
      const int q = tid >> 6, j = tid & 63;
      const double* a = tr + q * kThreads + j;
      double s4 = 0.0;
#pragma unroll
      for (int k = 0; k < kThreads / 64; k += 2) s4 += a[64 * k] + a[64 * (k + 1)];
      tr[3 * kThreads + q * 64 + j] = s4;
    }
    __syncthreads();
    if (tid < 3 * 32) {
      const int q = tid >> 5, lane = tid & 31;
      const double* b = tr + 3 * kThreads + q * 64;
      double x = b[lane] + b[lane + 32];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) bc[q] = x;
    }
    __syncthreads();
    if (tid == 0) {
      double t[4] = {bc[0], bc[1], bc[2], 0.0};
      t[3] = (clock64() > deadline) ? 1.0 : 0.0;
      int bad = 0;
      if (G > 1) {
        const int par = bar_count & 1;
        double* slot = P.red + ((size_t)par * G + g) * 4;
        for (int i = 0; i < 4; ++i) slot[i] = t[i];
        __threadfence();
        atomicAdd(P.bar, 1u);
        ++bar_count;
        const unsigned target = (unsigned)G * (unsigned)bar_count;
        const long long lim = deadline + (1ll << 31);
        while (ld_acquire_u32(P.bar) < target) {
          if (ld_volatile_i32(P.abort_flag) || clock64() > lim) { bad = 1; break; }
        }
        if (bad) atomicExch(P.abort_flag, 1);
        ctl[2] = par;
      }
      for (int i = 0; i < 4; ++i) bc[i] = t[i];
      ctl[0] = bad;
    }
    __syncthreads();
    if (G > 1 && !ctl[0]) {
      // Group totals: thread (i, k) sums the slots k, k + L, ... of quantity
      // i with independent L2 loads (the barrier above acquired them), then L
      // partials per quantity are added in a fixed order.  The vector staging
      // buffers are free between sweeps.
      static_assert(kThreads % 4 == 0, "four quantities");
      constexpr int L = kThreads / 4;
      double* part = reinterpret_cast<double*>(sm + kSmVs);
      const int par = ctl[2];
      const int i = tid / L, k = tid % L;
      double acc = 0.0;
      for (int gg = k; gg < G; gg += L) acc += __ldcg(P.red + ((size_t)par * G + gg) * 4 + i);
      part[tid] = acc;
      __syncthreads();
      if (tid < 4) {
        double sum = 0.0;
        for (int kk = 0; kk < L; ++kk) sum += part[tid * L + kk];
        bc[tid] = sum;
      }
      __syncthreads();
    }
    for (int i = 0; i < 4; ++i) v[i] = bc[i];
    if (ctl[0]) fail = true;
    __syncthreads();
  }

  // ---- vector rows of a chunk ---------------------------------------------
  // The vector arrays a sweep reads for one chunk, in a fixed order; `own`
  // arrays cover the chunk's owned rows [r0, r1), the others [base, vend).
  struct VecPlan {
    const char *src0, *src1, *src2, *src3;
    int esz0, esz1, esz2, esz3;
    int own0, own1, own2, own3;
    int cnt;
    __device__ __forceinline__ void add(const void* ptr, int esz, int own) {
      const char* c = static_cast<const char*>(ptr);
      if (cnt == 0) { src0 = c; esz0 = esz; own0 = own; }
      else if (cnt == 1) { src1 = c; esz1 = esz; own1 = own; }
      else if (cnt == 2) { src2 = c; esz2 = esz; own2 = own; }
      else { src3 = c; esz3 = esz; own3 = own; }
      ++cnt;
    }
    __device__ __forceinline__ const char* src(int i) const { return i == 0 ? src0 : (i == 1 ? src1 : (i == 2 ? src2 : src3)); }
    __device__ __forceinline__ int esz(int i) const { return i == 0 ? esz0 : (i == 1 ? esz1 : (i == 2 ? esz2 : esz3)); }
    __device__ __forceinline__ int own(int i) const { return i == 0 ? own0 : (i == 1 ? own1 : (i == 2 ? own2 : own3)); }
  };

  template <int STG, int FIN, typename T>
  static __device__ __forceinline__ VecPlan vec_plan(const Sweep<T>& sw) {
    VecPlan v{};
    v.cnt = 0;
    if constexpr (STG == SV_P) {
      v.add(sw.z, sizeof(T), 0);
      if (!sw.first) v.add(sw.p_old, sizeof(T), 0);
    } else if constexpr (STG == SV_VEC || STG == SV_R_FIRST) {
      v.add(sw.src64, 8, 0);
    } else if constexpr (STG == SV_R_UPD) {
      v.add(sw.r_old, sizeof(T), 0);
      v.add(sw.q, sizeof(T), 0);
      v.add(sw.x, sizeof(T), 1);
      v.add(sw.p_in, sizeof(T), 1);
    } else if constexpr (STG == SV_R_X0) {
      v.add(sw.src64, 8, 0);
      v.add(sw.q, sizeof(T), 0);
    } else {
      v.add(sw.yprev, sizeof(T), 0);
    }
    if constexpr (FIN == FN_YJ) {
      if (sw.j > 1) v.add(sw.zv, sizeof(T), 1);
      if (sw.last) v.add(sw.rcur_for_dot, sizeof(T), 1);
    } else if constexpr (FIN == FN_R64) {
      v.add(sw.bsub, 8, 1);
    }
    return v;
  }

  // Can the plan be moved by bulk copies (16-byte aligned rows, fits a slot)?
  static __device__ __forceinline__ bool vec_plan_ok(const VecPlan& v, int n, int R, int k, int halo, int VSB) {
    int bytes = 0;
    for (int i = 0; i < v.cnt; ++i) {
      if ((reinterpret_cast<uintptr_t>(v.src(i)) & 15u) != 0) return false;
      if (((long long)n * v.esz(i)) % 16 != 0) return false;
      const int rows = v.own(i) ? R : R + halo + k;
      bytes += rows * n * v.esz(i);
    }
    return bytes <= VSB;
  }

  // leader thread: bulk-copy the vector rows [base, vend) / [r0, r1) of a chunk
  static __device__ __forceinline__ void issue_vec(const VecPlan& v, int n, int r0, int r1, int base, int vend,
                                                   char* dst, uint64_t* bar) {
    unsigned total = 0;
    for (int i = 0; i < v.cnt; ++i) total += (unsigned)((v.own(i) ? (r1 - r0) : (vend - base)) * n * v.esz(i));
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bar, total);
    unsigned off = 0;
    for (int i = 0; i < v.cnt; ++i) {
      const int rows = v.own(i) ? (r1 - r0) : (vend - base);
      const int row0 = v.own(i) ? r0 : base;
      const unsigned bytes = (unsigned)(rows * n * v.esz(i));
      bulk_g2s(dst + off, v.src(i) + (size_t)row0 * n * v.esz(i), bytes, bar);
      off += bytes;
    }
  }

  // ---- one sweep, software-pipelined ---------------------------------------
  // The float32 sweeps of the inner iteration (A, B1, B2 with their vector
  // rows staged by bulk copies, n % 4 == 0).  Phase c computes the block
  // products of chunk c, finalizes chunk c-1 (and carries its pushes) and
  // stages the vector rows of chunk c+1: three disjoint sets of buffers
  // (partials double-, vector rows triple-buffered, in the room the layout
  // reserves for float64), so one CTA barrier per chunk separates the phases
  // instead of two, and the three kinds of work overlap across warps.  A
  // chunk's vector slot lives until its finalize, one phase after its
  // staging: the ring runs four slots, three chunks ahead.
  template <int KIND, int STG, int FIN>
  __device__ __noinline__ void sweep_pipe(const Sweep<float> sw, double acc[4]) {
    static_assert(KIND == kKA || KIND == kKB1 || KIND == kKB2, "stored-block sweeps only");
    static_assert(STG == SV_P || STG == SV_R_UPD || STG == SV_Y, "vectorised staging only");
    static_assert(FIN == FN_Q || FIN == FN_Y0 || FIN == FN_YJ, "vectorised finalize only");
    constexpr int kHalo = (KIND == kKB2) ? 2 : 1;
    constexpr int k = kHalo;
    constexpr int kPB = 3 * kMaxChunkElems + 2 * kMaxBlock;  // part1 | part2 | push of one buffer
    static_assert(2 * kPB * 4 <= (3 * kMaxChunkElems + 2 * kMaxBlock) * 8, "partials fit the float64 layout");
    static_assert(3 * kVsElems * 4 <= 2 * kVsElems * 8, "vector rows fit the float64 layout");
    static_assert(kVS == 4, "a chunk's vector slot lives one phase past its staging");
    Producer q = producer();
    const int n = this->n, N = this->N, s = this->s, e = this->e;
    const int S = this->S, SB = this->SB, VSB = this->VSB;
    const long long dl = deadline + (1ll << 31);
    uint64_t* const full = this->full;
    uint64_t* const vbar = this->vbar;
    char* const stages = this->stages;
    char* const vring = this->vring;
    unsigned consumed = this->consumed, vissued = this->vissued, vcons = this->vcons;
    const unsigned vbase = vcons;  // every slot issued so far has been consumed
    const bool leader = (threadIdx.x == kLeaderTid);
    const int tid = threadIdx.x;
    const int ts = (tid + kThreads / 2) % kThreads;  // staging from the upper half of the CTA
    const int R = q.rows(KIND);
    const int bse = bs;
    const float inv_n = 1.0f / (float)n;
    float* ringb = reinterpret_cast<float*>(sm + kSmRing);  // [2][k][n] by chunk parity
    float* vs3 = reinterpret_cast<float*>(sm + kSmVs);      // [3][kVsElems]
    float* pbuf = reinterpret_cast<float*>(sm + kSmParts);  // [2][kPB]
    const float sgn = (KIND == kKB1) ? -1.f : 1.f;
    const int nc = (e - s + R - 1) / R;
    const VecPlan vp = vec_plan<STG, FIN, float>(sw);
    const float alpha = sw.alpha, beta = sw.beta, alpha_j = sw.alpha_j;
    const bool first = sw.first, m1 = sw.m1, last = sw.last;
    const int jpow = sw.j;
    Accum<float> acc0, acc1, acc2;
    auto chunk_rows = [&](int c, int& r0, int& r1, int& base, int& vend) {
      r0 = s + c * R;
      r1 = min(e, r0 + R);
      base = r0 - ((c == 0) ? min(kHalo, s) : 0);
      vend = min(N, r1 + k);
    };
    // the vector-ring copies come from lane 0 of the warp below the stage
    // producer's, so the two issues after a phase barrier do not queue on one thread
    const bool vleader = (threadIdx.x == kLeaderTid - 32);
    auto issue = [&](int c) {
      if (vleader) {
        int r0, r1, base, vend;
        chunk_rows(c, r0, r1, base, vend);
        const int slot = (int)((vbase + (unsigned)c) % kVS);
        issue_vec(vp, n, r0, r1, base, vend, vring + (size_t)slot * VSB, &vbar[slot]);
      }
      ++vissued;
    };
    // the vector arrays of chunk c inside its slot (staging arrays first)
    auto slot_arrays = [&](int c, int nr, int rows, const float*& a0, const float*& a1, const float*& a2,
                           const float*& a3) {
      const char* vslot = vring + (size_t)((vbase + (unsigned)c) % kVS) * VSB;
      const int rng = rows * n, ow = nr * n;
      const int b0 = (vp.cnt > 0) ? (vp.own0 ? ow : rng) * vp.esz0 : 0;
      const int b1 = (vp.cnt > 1) ? (vp.own1 ? ow : rng) * vp.esz1 : 0;
      const int b2 = (vp.cnt > 2) ? (vp.own2 ? ow : rng) * vp.esz2 : 0;
      a0 = reinterpret_cast<const float*>(vslot);
      a1 = reinterpret_cast<const float*>(vslot + b0);
      a2 = reinterpret_cast<const float*>(vslot + b0 + b1);
      a3 = reinterpret_cast<const float*>(vslot + b0 + b1 + b2);
    };
    // stage the vector rows [base, vend) of chunk c with the fused PCG updates
    auto stage = [&](int c, bool& ok) {
      int r0, r1, base, vend;
      chunk_rows(c, r0, r1, base, vend);
      const int nr = r1 - r0, h = r0 - base;
      const unsigned vi = vbase + (unsigned)c;
      ok = ok && mbar_wait(&vbar[vi % kVS], (vi / kVS) & 1u, dl);
      ++vcons;
      const float *sv0, *sv1, *sv2, *sv3;
      slot_arrays(c, nr, vend - base, sv0, sv1, sv2, sv3);
      float* vs = vs3 + (c % 3) * kVsElems;
      const int nv = (vend - base) * n;
      for (int t = 4 * ts; t < nv; t += 4 * kThreads) {
        const int rr = qdiv(t, inv_n);
        const int a = t - rr * n;
        const int row = base + rr;
        const long long idx = (long long)row * n + a;
        const bool own = row >= r0 && row < r1;
        const int lo = t - h * n;
        float4 v;
        if constexpr (STG == SV_P) {
          const float4 zz = ld4f(sv0 + t);
          v = first ? zz : fma4(beta, ld4f(sv1 + t), zz);
          if (own) st4f(sw.p_cur + idx, v);
        } else if constexpr (STG == SV_R_UPD) {
          v = fma4(-alpha, ld4f(sv1 + t), ld4f(sv0 + t));
          if (own) {
            st4f(sw.r_cur + idx, v);
            st4f(sw.x + idx, fma4(alpha, ld4f(sv3 + lo), ld4f(sv2 + lo)));
            acc2.add(dot4f(v, v));
          }
        } else {
          v = ld4f(sv0 + t);
        }
        st4f(vs + t, v);
      }
    };
    // finalize the owned rows of chunk c (partials of phase c, pushes of the
    // row above from this chunk or the ring filled by chunk c-1)
    auto finalize = [&](int c) {
      int r0, r1, base, vend;
      chunk_rows(c, r0, r1, base, vend);
      const int nr = r1 - r0;
      const float *sv0, *sv1, *sv2, *sv3;
      slot_arrays(c, nr, vend - base, sv0, sv1, sv2, sv3);
      const float* vs = vs3 + (c % 3) * kVsElems;
      const float* part1 = pbuf + (c & 1) * kPB;
      const float* part2 = part1 + kMaxChunkElems;
      const float* push = part2 + kMaxChunkElems;
      const float* ring_in = ringb + ((c - 1) & 1) * (2 * kMaxBlock);
      const int ns = (STG == SV_P) ? (first ? 1 : 2) : ((STG == SV_R_UPD) ? 4 : 1);
      const int iz = ns, ir = ns + ((FIN == FN_YJ && jpow > 1) ? 1 : 0);
      const float* fz = (iz == 1) ? sv1 : ((iz == 2) ? sv2 : sv3);
      const float* fr = (ir == 1) ? sv1 : ((ir == 2) ? sv2 : sv3);
      const int nd = nr * n;
      for (int t = 4 * tid; t < nd; t += 4 * kThreads) {
        const int jj = qdiv(t, inv_n), a = t - jj * n;
        const int row = r0 + jj;
        const int src = row - k;
        float4 carry = make_float4(0.f, 0.f, 0.f, 0.f);
        if (src >= 0) carry = (src >= base) ? ld4f(push + (src - base) * n + a) : ld4f(ring_in + (src % k) * n + a);
        const float4 p1 = ld4f(part1 + t), p2 = ld4f(part2 + t);
        const float4 out = make_float4(p1.x + sgn * (p2.x + carry.x), p1.y + sgn * (p2.y + carry.y),
                                       p1.z + sgn * (p2.z + carry.z), p1.w + sgn * (p2.w + carry.w));
        const long long idx = (long long)row * n + a;
        const float4 vi = ld4f(vs + (row - base) * n + a);
        if constexpr (FIN == FN_Q) {
          st4f(sw.qout + idx, out);
          acc0.add(dot4f(vi, out));
        } else if constexpr (FIN == FN_Y0) {
          if (m1) {
            st4f(sw.zv + idx, out);
            acc1.add(dot4f(vi, out));
          } else {
            st4f(sw.y0 + idx, out);
            if constexpr (MF) st4f(sw.zv + idx, out);  // z starts at y0
          }
        } else {
          const float4 zprev = (jpow == 1) ? vi : ld4f(fz + t);
          const float4 zz = fma4(alpha_j, out, zprev);
          if (!last) st4f(sw.ynext + idx, out);
          st4f(sw.zv + idx, zz);
          if (last) acc1.add(dot4f(ld4f(fr + t), zz));
        }
      }
    };
    // the pushes of the last k source rows of chunk c, for chunk c+1
    auto carry = [&](int c) {
      int r0, r1, base, vend;
      chunk_rows(c, r0, r1, base, vend);
      const float* push = pbuf + (c & 1) * kPB + 2 * kMaxChunkElems;
      const float* ring_in = ringb + ((c - 1) & 1) * (2 * kMaxBlock);
      float* ring_out = ringb + (c & 1) * (2 * kMaxBlock);
      for (int t = (tid + kThreads - 64) % kThreads; t < k * n; t += kThreads) {
        const int w = qdiv(t, inv_n), a = t - w * n;
        const int src = r1 - k + w;
        if (src < 0) continue;
        ring_out[(src % k) * n + a] = (src >= base) ? push[(src - base) * n + a] : ring_in[(src % k) * n + a];
      }
    };

    for (int c = 0; c < min(kVS - 1, nc); ++c) issue(c);
    bool failed = false;
    {
      bool ok = true;
      if (nc > 0) stage(0, ok);
      if (__syncthreads_or(!ok)) {
        if (G > 1 && leader) atomicExch(P.abort_flag, 1);
        failed = true;
      }
    }
    for (int c = 0; c < nc && !failed; ++c) {
      int r0, r1, base, vend;
      chunk_rows(c, r0, r1, base, vend);
      const int nr = r1 - r0, h = r0 - base;
      const int st = consumed % S;
      const unsigned par = (consumed / S) & 1u;
      bool ok = mbar_wait(&full[st], par, dl);
      ++consumed;
      // products of chunk c (its vector rows were staged in the previous phase)
      const float* stg = reinterpret_cast<const float*>(stages + (size_t)st * SB);
      float* part1 = pbuf + (c & 1) * kPB;
      float* part2 = part1 + kMaxChunkElems;
      float* push = part2 + kMaxChunkElems;
      const float* vs = vs3 + (c % 3) * kVsElems;
      if (ok) {
        // block sizes of the OCP batches get unrolled products; every other n
        // takes the runtime-n form (an n = 48 specialization measured 2 %
        // slower on the 1024-instance batch: the instruction footprint of
        // the kernel, not its arithmetic, sets the cost of each variant)
        switch (n) {
          case 12: chunk_products<KIND, 12, float>(stg, R, bse, n, N, nr, h, r0, base, vs, part1, part2, push, nullptr, nullptr); break;
          case 24: chunk_products<KIND, 24, float>(stg, R, bse, n, N, nr, h, r0, base, vs, part1, part2, push, nullptr, nullptr); break;
          case 36: chunk_products<KIND, 36, float>(stg, R, bse, n, N, nr, h, r0, base, vs, part1, part2, push, nullptr, nullptr); break;
          default: chunk_products<KIND, 0, float>(stg, R, bse, n, N, nr, h, r0, base, vs, part1, part2, push, nullptr, nullptr); break;
        }
      }
      if (c > 0) {
        finalize(c - 1);
        carry(c - 1);
      }
      if (c + 1 < nc) stage(c + 1, ok);
      if (__syncthreads_or(!ok)) {
        if (G > 1 && leader) atomicExch(P.abort_flag, 1);
        failed = true;
        break;
      }
      q.step(leader);                          // the stage of chunk c is free
      if (c + kVS - 1 < nc) issue(c + kVS - 1);  // into the slot of chunk c-1
    }
    if (!failed && nc > 0) finalize(nc - 1);
    __syncthreads();
    this->consumed = consumed;
    this->vissued = vissued;
    this->vcons = vcons;
    store_producer(q);
    acc[0] += acc0.value();
    acc[1] += acc1.value();
    acc[2] += acc2.value();
    if (failed) fail = true;
  }

  // ---- one sweep -----------------------------------------------------------
  // KIND / STG / FIN are compile-time: each instantiation carries only the
  // staging and finalize code it uses.  The block products dispatch once per
  // chunk on n to compile-time block sizes (unrolled, vector loads).  The
  // vector rows each chunk reads arrive by bulk copies issued kVS-1
  // chunks ahead inside the sweep (they are final once the sweep starts).
  // All pipeline state is held in registers for the duration of the sweep.
  template <int KIND, int STG, int FIN, typename T>
  __device__ __noinline__ void sweep(const Sweep<T> sw, double acc[4]) {
    constexpr int kHalo = (KIND == kKB2 || KIND == kKB2G) ? 2 : 1;
    constexpr int k = (KIND == kKB2 || KIND == kKB2G) ? 2 : 1;
    if constexpr (sizeof(T) == 4 && kVS == 4 && (KIND == kKA || KIND == kKB1 || KIND == kKB2) &&
                  (STG == SV_P || STG == SV_R_UPD || STG == SV_Y) && (FIN == FN_Q || FIN == FN_Y0 || FIN == FN_YJ)) {
      if ((n & 3) == 0 && !sw.out_to_user &&
          vec_plan_ok(vec_plan<STG, FIN, T>(sw), n, geo(KIND).R, k, kHalo, VSB)) {
        sweep_pipe<KIND, STG, FIN>(sw, acc);
        return;
      }
    }
    Producer q = producer();
    const int n = this->n, N = this->N, s = this->s, e = this->e;
    const int S = this->S, SB = this->SB, VSB = this->VSB;
    const long long dl = deadline + (1ll << 31);
    uint64_t* const full = this->full;
    uint64_t* const vbar = this->vbar;
    char* const stages = this->stages;
    char* const vring = this->vring;
    unsigned consumed = this->consumed, vissued = this->vissued, vcons = this->vcons;
    const bool leader = (threadIdx.x == kLeaderTid);
    const int tid = threadIdx.x;
    // The staging of chunk c+1 starts from the upper half of the CTA while the
    // lower half still finalizes chunk c (at most kMaxChunkElems / 4 = 128
    // vectorised finalize tasks): the two touch different buffers and rows,
    // so they overlap instead of queuing on the same threads.
    const int ts = (tid + kThreads / 2) % kThreads;
    const int R = q.rows(KIND);
    const int bse = (KIND == kKA64) ? bs64 : bs;
    const float inv_n = 1.0f / (float)n;
    T* ringb = reinterpret_cast<T*>(sm + kSmRing);           // [2][k][n]
    T* vsb = reinterpret_cast<T*>(sm + kSmVs);               // [2][kVsElems]
    T* part1 = reinterpret_cast<T*>(sm + kSmParts);
    T* part2 = part1 + kMaxChunkElems;
    T* push = part2 + kMaxChunkElems;
    T* part3 = reinterpret_cast<T*>(sm + kSmFam);            // kKB2G only
    T* push1 = part3 + kMaxChunkElems;
    T* ring1b = push1 + kMaxChunkElems + 2 * kMaxBlock;      // [2][n]
    const T sgn = (KIND == kKB1) ? T(-1) : T(1);
    const int nc = (e - s + R - 1) / R;
    const VecPlan vp = vec_plan<STG, FIN, T>(sw);
    const bool va = vec_plan_ok(vp, n, R, k, kHalo, VSB);
    const bool vec4 = (sizeof(T) == 4) && va && ((n & 3) == 0);
    // staged inputs, copied to registers
    const T alpha = sw.alpha, beta = sw.beta, alpha_j = sw.alpha_j;
    const bool first = sw.first, m1 = sw.m1, last = sw.last, out_to_user = sw.out_to_user;
    const bool write_r = sw.write_r, zero_x = sw.zero_x;
    const int jpow = sw.j;
    const double scale = sw.scale;
    Accum<T> acc0, acc1, acc2;
    auto chunk_rows = [&](int c, int& r0, int& r1, int& base, int& vend) {
      r0 = s + c * R;
      r1 = min(e, r0 + R);
      base = r0 - ((c == 0) ? min(kHalo, s) : 0);
      vend = min(N, r1 + k);
    };
    if (va) {
      const int pre = min(kVS - 1, nc);
      for (int c = 0; c < pre; ++c) {
        if (leader) {
          int r0, r1, base, vend;
          chunk_rows(c, r0, r1, base, vend);
          const int slot = vissued % kVS;
          issue_vec(vp, n, r0, r1, base, vend, vring + (size_t)slot * VSB, &vbar[slot]);
        }
        ++vissued;
      }
    }
    bool failed = false;
    for (int c = 0; c < nc; ++c) {
      int r0, r1, base, vend;
      chunk_rows(c, r0, r1, base, vend);
      const int nr = r1 - r0;
      const int h = r0 - base;
      const int st = consumed % S;
      const unsigned par = (consumed / S) & 1u;
      const int buf = consumed & 1u;
      T* vs = vsb + buf * kVsElems;
      const T* ring_in = ringb + (buf ^ 1) * (2 * kMaxBlock);
      T* ring_out = ringb + buf * (2 * kMaxBlock);
      const T* ring1_in = ring1b + (buf ^ 1) * kMaxBlock;
      T* ring1_out = ring1b + buf * kMaxBlock;
      // 1. wait for the chunk's blocks and vector rows
      bool ok = mbar_wait(&full[st], par, dl);
      ++consumed;
      const char* vslot = vring + (size_t)(vcons % kVS) * VSB;
      if (va) {
        ok = ok && mbar_wait(&vbar[vcons % kVS], (vcons / kVS) & 1u, dl);
        ++vcons;
      }
      // byte offsets of the vector arrays inside the slot
      int voff1 = 0, voff2 = 0, voff3 = 0;
      {
        const int rng = (vend - base) * n, ow = nr * n;
        const int b0 = (vp.cnt > 0) ? (vp.own0 ? ow : rng) * vp.esz0 : 0;
        const int b1 = (vp.cnt > 1) ? (vp.own1 ? ow : rng) * vp.esz1 : 0;
        const int b2 = (vp.cnt > 2) ? (vp.own2 ? ow : rng) * vp.esz2 : 0;
        voff1 = b0;
        voff2 = b0 + b1;
        voff3 = b0 + b1 + b2;
      }
      const T* sv0 = reinterpret_cast<const T*>(vslot);
      const T* sv1 = reinterpret_cast<const T*>(vslot + voff1);
      const T* sv2 = reinterpret_cast<const T*>(vslot + voff2);
      const T* sv3 = reinterpret_cast<const T*>(vslot + voff3);
      const double* sd0 = reinterpret_cast<const double*>(vslot);
      // 2. stage the vector rows [base, vend) with the fused PCG updates
      const int nv = (vend - base) * n;
      bool staged4 = false;
      if constexpr (sizeof(T) == 4 && (STG == SV_P || STG == SV_R_UPD || STG == SV_Y)) {
        if (vec4) {  // 4 consecutive elements of one row per iteration
          staged4 = true;
          for (int t = 4 * ts; t < nv; t += 4 * kThreads) {
            const int rr = qdiv(t, inv_n);
            const int a = t - rr * n;
            const int row = base + rr;
            const long long idx = (long long)row * n + a;
            const bool own = row >= r0 && row < r1;
            const int lo = t - h * n;
            float4 v;
            if constexpr (STG == SV_P) {
              const float4 zz = ld4f(sv0 + t);
              v = first ? zz : fma4(beta, ld4f(sv1 + t), zz);
              if (own) st4f(sw.p_cur + idx, v);
            } else if constexpr (STG == SV_R_UPD) {
              v = fma4(-alpha, ld4f(sv1 + t), ld4f(sv0 + t));
              if (own) {
                st4f(sw.r_cur + idx, v);
                st4f(sw.x + idx, fma4(alpha, ld4f(sv3 + lo), ld4f(sv2 + lo)));
                acc2.add(dot4f(v, v));
              }
            } else {
              v = ld4f(sv0 + t);
            }
            st4f(vs + t, v);
          }
        }
      }
      if (!staged4)
      for (int t = ts; t < nv; t += kThreads) {
        const int rr = qdiv(t, inv_n);
        const int a = t - rr * n;
        const int row = base + rr;
        const long long idx = (long long)row * n + a;
        const bool own = row >= r0 && row < r1;
        const int lo = t - h * n;  // index among the owned rows
        T v;
        if constexpr (STG == SV_P) {
          const T zz = va ? sv0[t] : sw.z[idx];
          if (first) v = zz;
          else v = fma(beta, va ? sv1[t] : sw.p_old[idx], zz);
          if (own) sw.p_cur[idx] = v;
        } else if constexpr (STG == SV_VEC) {
          v = static_cast<T>(va ? sd0[t] : sw.src64[idx]);
        } else if constexpr (STG == SV_R_UPD) {
          v = fma(-alpha, va ? sv1[t] : sw.q[idx], va ? sv0[t] : sw.r_old[idx]);
          if (own) {
            sw.r_cur[idx] = v;
            sw.x[idx] = fma(alpha, va ? sv3[lo] : sw.p_in[idx], va ? sv2[lo] : sw.x[idx]);
            acc2.add(v * v);
          }
        } else if constexpr (STG == SV_R_FIRST) {
          v = static_cast<T>((va ? sd0[t] : sw.src64[idx]) * scale);
          if (own) {
            if (write_r) sw.r_cur[idx] = v;
            if (zero_x) sw.x[idx] = T(0);
            acc2.add(v * v);
          }
        } else if constexpr (STG == SV_R_X0) {
          v = static_cast<T>((va ? sd0[t] : sw.src64[idx]) - (double)(va ? sv1[t] : sw.q[idx]));
          if (own) {
            sw.r_cur[idx] = v;
            acc2.add(v * v);
          }
        } else {
          v = va ? sv0[t] : sw.yprev[idx];
        }
        vs[t] = v;
      }
      if (__syncthreads_or(!ok)) {
        if (G > 1 && leader) atomicExch(P.abort_flag, 1);
        failed = true;
        break;
      }
      // the vector slot of chunk c-1 is free now: prefetch chunk c + kVS - 1
      if (va && c + kVS - 1 < nc) {
        if (leader) {
          int pr0, pr1, pbase, pvend;
          chunk_rows(c + kVS - 1, pr0, pr1, pbase, pvend);
          const int slot = vissued % kVS;
          issue_vec(vp, n, pr0, pr1, pbase, pvend, vring + (size_t)slot * VSB, &vbar[slot]);
        }
        ++vissued;
      }
      // 3. block-vector products out of shared memory
      const T* stg = reinterpret_cast<const T*>(stages + (size_t)st * SB);
      switch (n) {
        case 12: chunk_products<KIND, 12, T>(stg, R, bse, n, N, nr, h, r0, base, vs, part1, part2, push, part3, push1); break;
        case 24: chunk_products<KIND, 24, T>(stg, R, bse, n, N, nr, h, r0, base, vs, part1, part2, push, part3, push1); break;
        case 36: chunk_products<KIND, 36, T>(stg, R, bse, n, N, nr, h, r0, base, vs, part1, part2, push, part3, push1); break;
        default: chunk_products<KIND, 0, T>(stg, R, bse, n, N, nr, h, r0, base, vs, part1, part2, push, part3, push1); break;
      }
      __syncthreads();
      if constexpr (KIND == kKJ) {
        // s_i = O_i v_{i+1} + O_{i-1}^T v_{i-1} (the push) into part1; the push
        // of the last row goes to the next chunk; then part2 = D^-1_i s_i
        for (int t = tid; t < nr * n; t += kThreads) {
          const int jj = qdiv(t, inv_n), a = t - jj * n;
          const int src = r0 + jj - 1;
          T carry = T(0);
          if (src >= 0) carry = (src >= base) ? push[(src - base) * n + a] : ring_in[a];
          part1[t] = part2[t] + carry;
        }
        for (int t = (tid + kThreads - 64) % kThreads; t < n; t += kThreads) ring_out[t] = push[(r1 - 1 - base) * n + t];
        __syncthreads();
        switch (n) {
          case 12: chunk_dinv<12, T>(stg, bse, n, nr, part1, part2); break;
          case 24: chunk_dinv<24, T>(stg, bse, n, nr, part1, part2); break;
          case 36: chunk_dinv<36, T>(stg, bse, n, nr, part1, part2); break;
          case 48: chunk_dinv<48, T>(stg, bse, n, nr, part1, part2); break;
          default: chunk_dinv<0, T>(stg, bse, n, nr, part1, part2); break;
        }
        __syncthreads();
      }
      // 4. the stage is free: refill it with the next predicted chunk
      q.step(leader);
      // 5. finalize owned rows
      const int nd = nr * n;
      // slot of the finalize-only arrays (after the staging arrays)
      const int ns = (STG == SV_P) ? (first ? 1 : 2) : ((STG == SV_R_UPD) ? 4 : ((STG == SV_R_X0) ? 2 : 1));
      const int iz = ns, ir = ns + ((FIN == FN_YJ && jpow > 1) ? 1 : 0);
      const T* fz = (iz == 1) ? sv1 : ((iz == 2) ? sv2 : sv3);
      const T* fr = (ir == 1) ? sv1 : ((ir == 2) ? sv2 : sv3);
      const double* fb = reinterpret_cast<const double*>((const char*)fz);
      bool fin4 = false;
      if constexpr (sizeof(T) == 4 && (FIN == FN_Q || FIN == FN_Y0 || FIN == FN_YJ || FIN == FN_T)) {
        if (vec4 && !out_to_user) {
          fin4 = true;
          for (int t = 4 * tid; t < nd; t += 4 * kThreads) {
            const int jj = qdiv(t, inv_n), a = t - jj * n;
            const int row = r0 + jj;
            const int src = row - k;
            float4 carry = make_float4(0.f, 0.f, 0.f, 0.f);
            if (src >= 0) carry = (src >= base) ? ld4f(push + (src - base) * n + a) : ld4f(ring_in + (src % k) * n + a);
            const float4 p1 = ld4f(part1 + t), p2 = ld4f(part2 + t);
            float4 out = make_float4(p1.x + sgn * (p2.x + carry.x), p1.y + sgn * (p2.y + carry.y),
                                     p1.z + sgn * (p2.z + carry.z), p1.w + sgn * (p2.w + carry.w));
            if constexpr (KIND == kKB2G) {  // the +-1 bands of H_ab
              const int src1 = row - 1;
              float4 c1 = make_float4(0.f, 0.f, 0.f, 0.f);
              if (src1 >= 0) c1 = (src1 >= base) ? ld4f(push1 + (src1 - base) * n + a) : ld4f(ring1_in + a);
              const float4 p3 = ld4f(part3 + t);
              out = make_float4(out.x + (p3.x + c1.x), out.y + (p3.y + c1.y), out.z + (p3.z + c1.z),
                                out.w + (p3.w + c1.w));
            }
            if constexpr (KIND == kKJ) out = make_float4(-p2.x, -p2.y, -p2.z, -p2.w);  // H_J v = -D^-1 s
            const long long idx = (long long)row * n + a;
            const float4 vi = ld4f(vs + (row - base) * n + a);
            if constexpr (FIN == FN_Q) {
              st4f(sw.qout + idx, out);
              acc0.add(dot4f(vi, out));
            } else if constexpr (FIN == FN_Y0) {
              if (m1) {
                st4f(sw.zv + idx, out);
                acc1.add(dot4f(vi, out));
              } else {
                st4f(sw.y0 + idx, out);
                if constexpr (MF) st4f(sw.zv + idx, out);  // z starts at y0
              }
            } else if constexpr (FIN == FN_T) {
              st4f(sw.ynext + idx, out);
            } else {
              const float4 zprev = (jpow == 1) ? vi : ld4f(fz + t);
              const float4 zz = fma4(alpha_j, out, zprev);
              if (!last) st4f(sw.ynext + idx, out);
              st4f(sw.zv + idx, zz);
              if (last) acc1.add(dot4f(ld4f(fr + t), zz));
            }
          }
        }
      }
      if (!fin4)
      for (int t = tid; t < nd; t += kThreads) {
        const int jj = qdiv(t, inv_n), a = t - jj * n;
        const int row = r0 + jj;
        const int src = row - k;
        T carry = T(0);
        if (src >= 0) carry = (src >= base) ? push[(src - base) * n + a] : ring_in[(src % k) * n + a];
        T out = part1[t] + sgn * (part2[t] + carry);
        if constexpr (KIND == kKB2G) {  // the +-1 bands of H_ab
          const int src1 = row - 1;
          T c1 = T(0);
          if (src1 >= 0) c1 = (src1 >= base) ? push1[(src1 - base) * n + a] : ring1_in[a];
          out += part3[t] + c1;
        }
        if constexpr (KIND == kKJ) out = -part2[t];  // H_J v = -D^-1 s
        const long long idx = (long long)row * n + a;
        const T vi = vs[(row - base) * n + a];
        if constexpr (FIN == FN_Q) {
          sw.qout[idx] = out;
          acc0.add(vi * out);
        } else if constexpr (FIN == FN_OUT64) {
          sw.out64[idx] = (double)out;
        } else if constexpr (FIN == FN_R64) {
          const double r = (va ? fb[t] : sw.bsub[idx]) - (double)out;
          sw.r64[idx] = r;
          acc0.add(r * r);
        } else if constexpr (FIN == FN_Y0) {
          if (m1) {
            if (out_to_user) sw.out64[idx] = (double)out;
            else sw.zv[idx] = out;
            acc1.add(vi * out);
          } else {
            sw.y0[idx] = out;
            if constexpr (MF) sw.zv[idx] = out;  // z starts at y0
          }
        } else if constexpr (FIN == FN_T) {
          sw.ynext[idx] = out;
        } else {  // FN_YJ
          const T zprev = (jpow == 1) ? vi : (va ? fz[t] : sw.zv[idx]);
          const T zz = fma(alpha_j, out, zprev);
          if (!last) sw.ynext[idx] = out;
          if (last && out_to_user) sw.out64[idx] = (double)zz;
          else sw.zv[idx] = zz;
          if (last) acc1.add((va ? fr[t] : sw.rcur_for_dot[idx]) * zz);
        }
      }
      // 6. carry the pushes of the last k source rows into the other ring
      //    buffer (read by the next chunk after its barriers); kKB2G also
      //    carries push1 of its last row
      constexpr int kc = (KIND == kKB2G) ? k + 1 : ((KIND == kKJ) ? 0 : k);  // kKJ carried before its D^-1 phase
      for (int t = (tid + kThreads - 64) % kThreads; t < kc * n; t += kThreads) {  // threads 64.. (idle in finalize)
        const int w = qdiv(t, inv_n), a = t - w * n;
        if (KIND == kKB2G && w == k) {
          ring1_out[a] = push1[(r1 - 1 - base) * n + a];
          continue;
        }
        const int src = r1 - k + w;
        if (src < 0) continue;
        ring_out[(src % k) * n + a] = (src >= base) ? push[(src - base) * n + a] : ring_in[(src % k) * n + a];
      }
    }
    this->consumed = consumed;
    this->vissued = vissued;
    this->vcons = vcons;
    store_producer(q);
    acc[0] += acc0.value();
    acc[1] += acc1.value();
    acc[2] += acc2.value();
    if (failed) fail = true;
  }

  // ---- vector-only passes over the owned rows ------------------------------
  __device__ double vpass_norm2(const double* v) {
    double acc = 0.0;
    for (long long i = (long long)s * n + tid; i < (long long)e * n; i += kThreads) acc += v[i] * v[i];
    return acc;
  }
};

// ---------------------------------------------------------------------------
// The kernel.
// ---------------------------------------------------------------------------
template <typename MT, int VAR>
__device__ void solve_instance(Solver<MT, VAR>& Sv, int inst_id);

template <typename MT, int VAR>
__global__ void __launch_bounds__(kThreads, 1) bt_persistent_kernel(const __grid_constant__ KParams P) {
  extern __shared__ __align__(128) char smem[];
  Solver<MT, VAR> Sv(P, smem);
  if (threadIdx.x == kLeaderTid) {
    for (int i = 0; i < P.stages; ++i) mbar_init(&Sv.full[i], 1);
    for (int i = 0; i < kVecSlots; ++i) mbar_init(&Sv.vbar[i], 1);
    fence_mbar_init();
  }
  __syncthreads();
  int* ctl = reinterpret_cast<int*>(smem + kSmCtl);
  Sv.G = P.G;
  Sv.g = (P.G > 1) ? (int)blockIdx.x : 0;
  for (;;) {
    int inst;
    if (P.G > 1) {
      inst = 0;
    } else {
      if (threadIdx.x == 0) ctl[1] = atomicAdd(P.queue, 1);
      __syncthreads();
      const int idx = ctl[1];
      __syncthreads();
      if (idx >= P.B) break;
      inst = P.order[idx];
    }
    solve_instance<MT, VAR>(Sv, inst);
    if (P.G > 1) break;
  }
}

template <typename MT, int VAR>
__device__ void solve_instance(Solver<MT, VAR>& Sv, int inst_id) {
  constexpr bool GEN = Solver<MT, VAR>::GEN;
  constexpr bool MF = Solver<MT, VAR>::MF;
  const KParams& P = Sv.P;
  const InstDesc d = P.inst[inst_id];
  const int tid = threadIdx.x;
  Sv.N = d.N;
  Sv.n = d.n;
  Sv.vec = d.vec;
  Sv.bs = (sizeof(MT) == 4) ? d.bs32 : d.bs64;
  Sv.bs64 = d.bs64;
  if (Sv.G > 1) {
    Sv.s = (int)((long long)Sv.g * d.N / Sv.G);
    Sv.e = (int)((long long)(Sv.g + 1) * d.N / Sv.G);
  } else {
    Sv.s = 0;
    Sv.e = d.N;
  }
  Sv.fail = false;
  Sv.status = kOK;
  Sv.deadline = clock64() + P.budget;
  const int n = d.n, m = P.m;
  if (sizeof(MT) == 4) {
    const long long o = d.off32;
    Sv.mats[0] = (const MT*)(P.D32 + o); Sv.mats[1] = (const MT*)(P.O32 + o);
    Sv.mats[2] = (const MT*)(P.Dinv32 + o); Sv.mats[3] = (const MT*)(P.E32 + o);
    Sv.mats[4] = (const MT*)(P.Hd32 + o); Sv.mats[5] = (const MT*)(P.Hu32 + o);
    Sv.mats[6] = (const MT*)(P.Hl32 + o);
    if constexpr (GEN) {
      Sv.mats[7] = (const MT*)(P.F32 + o);
      Sv.mats[8] = (const MT*)(P.K32 + o);
    }
  } else {
    const long long o = d.off64;
    Sv.mats[0] = (const MT*)(P.D64 + o); Sv.mats[1] = (const MT*)(P.O64 + o);
    Sv.mats[2] = (const MT*)(P.Dinv64 + o); Sv.mats[3] = (const MT*)(P.E64 + o);
    Sv.mats[4] = (const MT*)(P.Hd64 + o); Sv.mats[5] = (const MT*)(P.Hu64 + o);
    Sv.mats[6] = (const MT*)(P.Hl64 + o);
    if constexpr (GEN) {
      Sv.mats[7] = (const MT*)(P.F64 + o);
      Sv.mats[8] = (const MT*)(P.K64 + o);
    }
  }
  Sv.mats64[0] = P.D64 + d.off64;
  Sv.mats64[1] = P.O64 + d.off64;
  Sv.set_chunk_counts();

  // workspace slot
  const int slot = (Sv.G > 1) ? 0 : (int)blockIdx.x;
  char* wsb = P.ws + (size_t)slot * P.ws_stride;
  const long long V = P.ws_vec;
  MT* wv = reinterpret_cast<MT*>(wsb);
  MT* x_in = wv + 0 * V;
  MT* rb[2] = {wv + 1 * V, wv + 2 * V};
  MT* pb[2] = {wv + 3 * V, wv + 4 * V};
  MT* q = wv + 5 * V;
  MT* y0 = wv + 6 * V;
  MT* ya = wv + 7 * V;
  MT* yb = wv + 8 * V;
  MT* z = wv + 9 * V;
  double* r64 = reinterpret_cast<double*>(wsb + (size_t)10 * V * sizeof(MT));

  const double* bu = P.bvec + d.vec;  // user input vector
  double* xu = P.xvec + d.vec;        // user output vector
  const bool mixed = P.mixed != 0;

  // pattern of the inner iteration: A, B1, B2 x (m-1)

  double acc[4];
  auto zero_acc = [&]() { acc[0] = acc[1] = acc[2] = acc[3] = 0.0; };
  // PCG step scalars: the float32 inner iteration uses them rounded to float,
  // so by default it divides in float32 (a float64 division is a dozen
  // float64 instructions on every thread); with P.scal64 (the strict float64
  // split) and on the float64 path it divides in float64.
  const bool scal64 = P.scal64 != 0;
  auto sdiv = [scal64](double a, double b) -> double {
    if constexpr (sizeof(MT) == 4) return scal64 ? a / b : (double)__fdiv_rn((float)a, (float)b);
    else return a / b;
  };

  // Apply z = M^-1 rhs into the inner vectors (or to the user array).
  // Runs B1 then B2 x (m-1); rz accumulates in acc[1] of the last sweep.
  // rhs given by (src64, scale) when first_from_user, else r already staged
  // through SV_R_UPD by the caller.
  // Matrix-free variant: H_opt y = H_J (H_J y); the first H_J goes to q
  // (free between B1 and the next A), the second finalizes y_j.  B1 has
  // written z = y0 already, so every y_j step adds to z (j > 1 form).
  auto precond_sweeps_after_b1 = [&](MT* rcur, bool to_user) {
    for (int j = 1; j < m; ++j) {
      const MT* yp = (j == 1) ? y0 : ((j - 1) % 2 == 1 ? ya : yb);
      if constexpr (MF) {
        Sweep<MT> st = {};
        st.kind = kKJ; st.stg = SV_Y; st.fin = FN_T; st.sgn = MT(1);
        st.yprev = yp; st.ynext = q;
        zero_acc();
        Sv.template sweep<kKJ, SV_Y, FN_T>(st, acc);
        Sv.group_reduce(acc);
        if (Sv.fail) return;
        yp = q;
      }
      Sweep<MT> sw = {};
      sw.kind = Solver<MT, VAR>::kHK; sw.stg = SV_Y; sw.fin = FN_YJ; sw.sgn = MT(1);
      sw.yprev = yp;
      sw.ynext = (j % 2 == 1) ? ya : yb;
      sw.zv = z; sw.j = MF ? j + 1 : j; sw.m = m; sw.alpha_j = (MT)P.alpha[j]; sw.last = (j == m - 1);
      sw.rcur_for_dot = rcur; sw.out_to_user = to_user; sw.out64 = xu;
      zero_acc();
      Sv.template sweep<Solver<MT, VAR>::kHK, SV_Y, FN_YJ>(sw, acc);
      Sv.group_reduce(acc);
      if (Sv.fail) return;
    }
  };

  int iters_total = 0, outer = 0;
  double resid = 0.0, errv = 0.0;

  if (P.op == kOpSpmv64 || (P.op == kOpSpmv32 && sizeof(MT) == 8)) {
    Sv.restart(kKA64, 1, 0);
    Sweep<double> sw = {};
    sw.kind = kKA64; sw.stg = SV_VEC; sw.fin = FN_OUT64; sw.sgn = 1.0;
    sw.src64 = bu; sw.out64 = xu;
    zero_acc();
    Sv.template sweep<kKA64, SV_VEC, FN_OUT64>(sw, acc);
    Sv.group_reduce(acc);
  } else if (P.op == kOpSpmv32) {
    Sv.restart(kKA, 1, 0);
    Sweep<MT> sw = {};
    sw.kind = kKA; sw.stg = SV_VEC; sw.fin = FN_OUT64; sw.sgn = MT(1);
    sw.src64 = bu; sw.out64 = xu;
    zero_acc();
    Sv.template sweep<kKA, SV_VEC, FN_OUT64>(sw, acc);
    Sv.group_reduce(acc);
  } else if (P.op == kOpApply) {
    Sv.restart(kKA, 2 + Solver<MT, VAR>::kHPS * (m - 1), 1);
    Sweep<MT> sw = {};
    sw.kind = kKB1; sw.stg = SV_R_FIRST; sw.fin = FN_Y0; sw.sgn = MT(-1);
    sw.src64 = bu; sw.scale = 1.0; sw.r_cur = rb[0]; sw.write_r = true; sw.zero_x = false;
    sw.y0 = y0; sw.m1 = (m == 1); sw.out_to_user = true; sw.out64 = xu; sw.zv = z;
    zero_acc();
    Sv.template sweep<kKB1, SV_R_FIRST, FN_Y0>(sw, acc);
    Sv.group_reduce(acc);
    if (!Sv.fail) precond_sweeps_after_b1(rb[0], true);
  } else {
    // ------------------------------ SOLVE ------------------------------
    // Inner PCG on S d = rhs (rhs from src64 * scale or b - S x0), textbook
    // form; returns iterations, sets status, leaves the solution in xvec.
    // optional history: iteration it_base + k - 1 of this instance gets the
    // relative residual of this inner solve, alpha_k and beta_k (Lanczos
    // coefficients of the preconditioned operator)
    double* const hist = (P.hist && tid == 0 && Sv.g == 0) ? P.hist + (size_t)inst_id * P.hist_len * 3 : nullptr;
    auto record = [&](int idx, int field, double v) {
      if (hist && idx >= 0 && idx < P.hist_len) hist[(size_t)idx * 3 + field] = v;
    };
    auto inner_pcg = [&](const double* src64, double scale, MT* xv, bool from_x0, double tol_rel,
                         int maxit, int& it_out, int& st_out, double& rr_out, int it_base) {
      it_out = 0;
      st_out = kOK;
      // initial residual and z0 = M^-1 r0
      Sv.restart(kKA, 2 + Solver<MT, VAR>::kHPS * (m - 1), from_x0 ? 0 : 1);
      if (from_x0) {
        Sweep<MT> sa = {};
        sa.kind = kKA; sa.stg = SV_VEC; sa.fin = FN_Q; sa.sgn = MT(1);
        sa.src64 = reinterpret_cast<const double*>(xv);  // float64 path only
        sa.qout = q;
        zero_acc();
        Sv.template sweep<kKA, SV_VEC, FN_Q>(sa, acc);
        Sv.group_reduce(acc);
        if (Sv.fail) { st_out = kErrTimeout; return; }
      }
      Sweep<MT> s1 = {};
      s1.kind = kKB1; s1.fin = FN_Y0; s1.sgn = MT(-1);
      s1.r_cur = rb[0]; s1.write_r = true; s1.x = xv;
      if (from_x0) { s1.stg = SV_R_X0; s1.src64 = src64; s1.q = q; s1.zero_x = false; }
      else { s1.stg = SV_R_FIRST; s1.src64 = src64; s1.scale = scale; s1.zero_x = true; }
      s1.y0 = y0; s1.m1 = (m == 1); s1.out_to_user = false; s1.zv = z;
      zero_acc();
      if (from_x0) Sv.template sweep<kKB1, SV_R_X0, FN_Y0>(s1, acc);
      else Sv.template sweep<kKB1, SV_R_FIRST, FN_Y0>(s1, acc);
      Sv.group_reduce(acc);
      if (Sv.fail) { st_out = kErrTimeout; return; }
      if (acc[3] > 0) { st_out = kErrTimeout; return; }
      double rr = acc[2], rz = acc[1];
      rr_out = rr;
      if (!isfinite(rr)) { st_out = kErrNonfinite; return; }
      // rhs norm: for the plain start r0 = rhs
      double nrhs;
      if (from_x0) {
        // ||b|| for the stopping rule
        double t[4] = {Sv.vpass_norm2(src64), 0, 0, 0};
        Sv.group_reduce(t);
        nrhs = sqrt(t[0]);
      } else {
        nrhs = sqrt(rr);
      }
      if (nrhs == 0.0) { return; }  // x = 0 already
      // ||r|| <= tol ||rhs||, squared (no per-iteration square root)
      const double thr2 = (tol_rel * nrhs) * (tol_rel * nrhs);
      if (rr <= thr2) { return; }
      if (m > 1) {
        precond_sweeps_after_b1(rb[0], false);
        if (Sv.fail) { st_out = kErrTimeout; return; }
        rz = acc[1];
      }
      double rho = rz;
      double beta = 0.0;
      for (int k = 1;; ++k) {
        if (k > maxit) { st_out = kErrNoConv; it_out = maxit; return; }
        // A: q = S p, p = z + beta p_old
        Sweep<MT> sa = {};
        sa.kind = kKA; sa.stg = SV_P; sa.fin = FN_Q; sa.sgn = MT(1);
        sa.z = z; sa.p_old = pb[(k + 1) & 1]; sa.p_cur = pb[k & 1];
        sa.beta = (MT)beta; sa.first = (k == 1); sa.qout = q;
        zero_acc();
        Sv.template sweep<kKA, SV_P, FN_Q>(sa, acc);
        Sv.group_reduce(acc);
        if (Sv.fail || acc[3] > 0) { st_out = kErrTimeout; it_out = k - 1; return; }
        const double pq = acc[0];
        if (!isfinite(pq)) { st_out = kErrNonfinite; it_out = k - 1; return; }
        if (!(pq > 0.0)) { st_out = kErrBreakdown; it_out = k - 1; errv = pq; return; }
        const double alpha = sdiv(rho, pq);
        record(it_base + k - 1, 1, alpha);
        record(it_base + k - 1, 2, 0.0);
        // B1: r -= alpha q, x += alpha p, y0 = G r
        Sweep<MT> sb = {};
        sb.kind = kKB1; sb.stg = SV_R_UPD; sb.fin = FN_Y0; sb.sgn = MT(-1);
        sb.alpha = (MT)alpha; sb.r_old = rb[(k + 1) & 1]; sb.r_cur = rb[k & 1]; sb.q = q;
        sb.x = xv; sb.p_in = pb[k & 1];
        sb.y0 = y0; sb.m1 = (m == 1); sb.out_to_user = false; sb.zv = z;
        zero_acc();
        Sv.template sweep<kKB1, SV_R_UPD, FN_Y0>(sb, acc);
        Sv.group_reduce(acc);
        if (Sv.fail || acc[3] > 0) { st_out = kErrTimeout; it_out = k; return; }
        rr = acc[2];
        rr_out = rr;
        it_out = k;
        record(it_base + k - 1, 0, sqrt(rr) / nrhs);
        if (!isfinite(rr)) { st_out = kErrNonfinite; return; }
        if (rr <= thr2) return;
        if (m > 1) {
          precond_sweeps_after_b1(rb[k & 1], false);
          if (Sv.fail) { st_out = kErrTimeout; return; }
        }
        const double rz_new = acc[1];
        beta = sdiv(rz_new, rho);
        record(it_base + k - 1, 2, beta);
        rho = rz_new;
      }
    };

    if (!mixed) {
      // float64 path: PCG directly on the user vectors
      int it, st;
      double rr;
      MT* xv = reinterpret_cast<MT*>(xu);
      inner_pcg(bu, 1.0, xv, P.use_x0 != 0, P.tol, P.maxit, it, st, rr, 0);
      iters_total = it;
      Sv.status = st;
      double t[4] = {Sv.vpass_norm2(bu), 0, 0, 0};
      Sv.group_reduce(t);
      const double nb = sqrt(t[0]);
      resid = nb > 0 ? sqrt(rr) / nb : 0.0;
      if (st == kErrBreakdown) resid = errv;
    } else {
      // mixed: float32 inner PCG inside float64 iterative refinement
      double t[4] = {Sv.vpass_norm2(bu), 0, 0, 0};
      Sv.group_reduce(t);
      const double nb = sqrt(t[0]);
      const double tol = P.tol;
      int st = kOK;
      if (!isfinite(nb)) {
        st = kErrNonfinite;
      } else if (nb == 0.0) {
        for (long long i = (long long)Sv.s * n + tid; i < (long long)Sv.e * n; i += kThreads) xu[i] = 0.0;
        resid = 0.0;
      } else {
        if (!P.use_x0)
          for (long long i = (long long)Sv.s * n + tid; i < (long long)Sv.e * n; i += kThreads) xu[i] = 0.0;
        double nr = nb;
        for (outer = 0;; ++outer) {
          const bool have_r64 = (outer > 0) || P.use_x0;
          if (have_r64) {
            Sv.restart(kKA64, 1, 0);
            Sweep<double> sw = {};
            sw.kind = kKA64; sw.stg = SV_VEC; sw.fin = FN_R64; sw.sgn = 1.0;
            sw.src64 = xu; sw.bsub = bu; sw.r64 = r64;
            zero_acc();
            Sv.template sweep<kKA64, SV_VEC, FN_R64>(sw, acc);
            Sv.group_reduce(acc);
            if (Sv.fail || acc[3] > 0) { st = kErrTimeout; break; }
            nr = sqrt(acc[0]);
            if (!isfinite(nr)) { st = kErrNonfinite; break; }
          }
          resid = nr / nb;
          if (nr <= tol * nb) { st = kOK; break; }
          if (outer >= P.max_outer || iters_total >= P.maxit) { st = kErrNoConv; break; }
          // inner tolerance: the caller's, else sqrt(tol) in [1e-6, 1e-4] --
          // two refinement steps of sqrt(tol) each reach tol, and the float32
          // inner iteration resolves ~1e-6 at best
          double t_in = P.tol_inner > 0.0 ? P.tol_inner : fmin(1e-4, fmax(1e-6, sqrt(tol)));
          const double need = 0.5 * tol * nb / nr;
          if (need > t_in) t_in = need;
          if (t_in > 0.5) t_in = 0.5;
          int it, ist;
          double rr;
          inner_pcg(have_r64 ? r64 : bu, 1.0 / nr, x_in, false, t_in, P.maxit - iters_total, it, ist, rr,
                    iters_total);
          iters_total += it;
          if (ist == kErrBreakdown || ist == kErrNonfinite || ist == kErrTimeout) { st = ist; break; }
          // x += nr * d over the owned rows, then make it visible to the group
          for (long long i = (long long)Sv.s * n + tid; i < (long long)Sv.e * n; i += kThreads)
            xu[i] = fma(nr, (double)x_in[i], xu[i]);
          double tt[4] = {0, 0, 0, 0};
          Sv.group_reduce(tt);
          if (Sv.fail) { st = kErrTimeout; break; }
        }
      }
      Sv.status = st;
    }
  }
  Sv.flush();
  if (Sv.fail) Sv.status = kErrTimeout;
  if (tid == 0 && Sv.g == 0 && P.op == kOpSolve) {
    P.iters[inst_id] = iters_total;
    P.status[inst_id] = Sv.status;
    P.outer[inst_id] = outer;
    P.resid[inst_id] = resid;
    P.errval[inst_id] = errv;
  }
}

}  // namespace bt
