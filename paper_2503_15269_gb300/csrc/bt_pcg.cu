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
#include "bt_common.cuh"

namespace bt {

enum Kind : int { kKA = 0, kKB1 = 1, kKB2 = 2, kKA64 = 3 };
enum StageMode : int { SV_P = 0, SV_VEC = 1, SV_R_UPD = 2, SV_R_FIRST = 3, SV_R_X0 = 4, SV_Y = 5 };
enum FinMode : int { FN_Q = 0, FN_OUT64 = 1, FN_R64 = 2, FN_Y0 = 3, FN_YJ = 4 };

// Per-kind chunk geometry.
struct Geo {
  int R;      // owned rows per chunk
  int halo;   // push-only rows before a CTA range start
  int k;      // push distance (1 for S and G, 2 for H)
  int narr;   // block arrays in the chunk
};

__device__ __forceinline__ Geo geo_of(int kind, int stage_bytes, int bs_bytes, int n) {
  Geo g;
  const int slots = stage_bytes / bs_bytes;
  if (kind == kKB2) {
    g.R = (slots - 2) / 3; g.halo = 2; g.k = 2; g.narr = 3;
  } else {
    g.R = (slots - 1) / 2; g.halo = 1; g.k = 1; g.narr = 2;
  }
  const int cap = kMaxChunkElems / n;
  if (g.R > cap) g.R = cap;
  if (g.R < 1) g.R = 1;
  return g;
}

// Smem carve-up (bytes).  Fixed part first, then the stages (128-aligned).
constexpr int kSmCtl = 0;                               // ints
constexpr int kSmRed = 128;                             // double [8 warps][4]
constexpr int kSmBc = kSmRed + 8 * 4 * 8;               // double bcast[8]
constexpr int kSmRing = kSmBc + 8 * 8;                  // T ring[2][64]
constexpr int kSmVs = kSmRing + 2 * kMaxBlock * 8;      // T vs[kMaxChunkElems + 4*64]
constexpr int kSmParts = kSmVs + (kMaxChunkElems + 4 * kMaxBlock) * 8;  // T p1[512], p2[512], push[512+128]
constexpr int kSmFull = kSmParts + (3 * kMaxChunkElems + 2 * kMaxBlock) * 8;  // uint64 full[kMaxStages]
constexpr int kSmStages = ((kSmFull + kMaxStages * 8 + 127) / 128) * 128;

__host__ __device__ constexpr int smem_fixed_bytes() { return kSmStages; }

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

template <typename MT>
struct Solver {
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
  int pat[kMaxM + 2];
  int pat_len, p_slot, p_chunk;
  const double* mats64[7];
  const MT* mats[7];
  int bs, bs64;

  __device__ Solver(const KParams& P_, char* sm_) : P(P_), sm(sm_) {
    tid = threadIdx.x;
    S = P.stages;
    SB = P.stage_bytes;
    full = reinterpret_cast<uint64_t*>(sm + kSmFull);
    stages = sm + kSmStages;
    issued = consumed = 0;
    bar_count = 0;
  }

  // ---- chunk geometry ----------------------------------------------------
  __device__ int bsb_of(int kind) const { return kind == kKA64 ? bs64 * 8 : bs * (int)sizeof(MT); }
  __device__ Geo geo(int kind) const { return geo_of(kind, SB, bsb_of(kind), n); }
  __device__ int nchunks(int kind) const {
    Geo gg = geo(kind);
    return (e - s + gg.R - 1) / gg.R;
  }

  // ---- producer (thread 0 only) ------------------------------------------
  __device__ void issue(int kind, int c) {
    const Geo gg = geo(kind);
    const int r0 = s + c * gg.R;
    const int r1 = min(e, r0 + gg.R);
    const int h = (c == 0) ? min(gg.halo, s) : 0;
    const int bsb = bsb_of(kind);
    const int st = issued % S;
    char* dst = stages + (size_t)st * SB;
    uint64_t* bar = &full[st];
    const int nr = r1 - r0;
    unsigned total;
    if (kind == kKB2) total = (unsigned)(3 * nr + h) * bsb;
    else total = (unsigned)(2 * nr + h) * bsb;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bar, total);
    if (kind == kKA64) {
      const double* D = mats64[0];
      const double* O = mats64[1];
      bulk_g2s(dst, D + (size_t)r0 * bs64, nr * bsb, bar);
      bulk_g2s(dst + (size_t)gg.R * bsb, O + (size_t)(r0 - h) * bs64, (nr + h) * bsb, bar);
    } else {
      const MT* A0 = kind == kKA ? mats[0] : (kind == kKB1 ? mats[2] : mats[4]);
      const MT* A1 = kind == kKA ? mats[1] : (kind == kKB1 ? mats[3] : mats[5]);
      bulk_g2s(dst, A0 + (size_t)r0 * bs, nr * bsb, bar);
      if (kind == kKB2) {
        bulk_g2s(dst + (size_t)gg.R * bsb, A1 + (size_t)r0 * bs, nr * bsb, bar);
        bulk_g2s(dst + (size_t)2 * gg.R * bsb, mats[6] + (size_t)(r0 - h) * bs, (nr + h) * bsb, bar);
      } else {
        bulk_g2s(dst + (size_t)gg.R * bsb, A1 + (size_t)(r0 - h) * bs, (nr + h) * bsb, bar);
      }
    }
    ++issued;
  }

  __device__ void issue_next() {
    // thread 0: issue the chunk at the producer cursor, then advance it.
    const int kind = pat[p_slot];
    issue(kind, p_chunk);
    if (++p_chunk >= nchunks(kind)) {
      p_chunk = 0;
      p_slot = (p_slot + 1) % pat_len;
    }
  }

  // Drain every chunk in flight (bounded) so that the ring is idle.
  __device__ void flush() {
    bool ok = true;
    while (consumed < issued) {
      const int st = consumed % S;
      const unsigned par = (consumed / S) & 1u;
      if (ok && !mbar_wait(&full[st], par, deadline + (1ll << 31))) ok = false;
      ++consumed;
    }
    __syncthreads();
    if (!ok) fail = true;
  }

  // Start a new predicted sweep sequence: pattern `p[0..len)`, starting slot.
  __device__ void restart(const int* p, int len, int start_slot) {
    flush();
    pat_len = len;
    for (int i = 0; i < len; ++i) pat[i] = p[i];
    p_slot = start_slot;
    p_chunk = 0;
    if (tid == 0) {
      for (int i = 0; i < S; ++i) issue_next();
    } else {
      // keep the uniform copies of the cursor in step with thread 0
      for (int i = 0; i < S; ++i) {
        ++issued;
        if (++p_chunk >= nchunks(pat[p_slot])) { p_chunk = 0; p_slot = (p_slot + 1) % pat_len; }
      }
    }
  }

  __device__ void advance_producer_after_release() {
    if (tid == 0) {
      issue_next();
    } else {
      ++issued;
      if (++p_chunk >= nchunks(pat[p_slot])) { p_chunk = 0; p_slot = (p_slot + 1) % pat_len; }
    }
  }

  // ---- reductions & group barrier ----------------------------------------
  // Reduce 4 per-thread partials over the CTA, then over the group (fixed
  // order, so results are bitwise reproducible).  v[3] carries a timeout flag.
  __device__ void group_reduce(double v[4]) {
    if (fail) return;
    double* red = reinterpret_cast<double*>(sm + kSmRed);
    double* bc = reinterpret_cast<double*>(sm + kSmBc);
    int* ctl = reinterpret_cast<int*>(sm + kSmCtl);
    const int lane = tid & 31, w = tid >> 5;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      double x = v[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) red[w * 4 + i] = x;
    }
    __syncthreads();
    if (tid == 0) {
      double t[4] = {0, 0, 0, 0};
      for (int ww = 0; ww < kThreads / 32; ++ww)
        for (int i = 0; i < 4; ++i) t[i] += red[ww * 4 + i];
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
        if (!bad) {
          for (int i = 0; i < 4; ++i) t[i] = 0.0;
          for (int gg = 0; gg < G; ++gg) {
            const volatile double* o = P.red + ((size_t)par * G + gg) * 4;
            for (int i = 0; i < 4; ++i) t[i] += o[i];
          }
        } else {
          atomicExch(P.abort_flag, 1);
        }
      }
      for (int i = 0; i < 4; ++i) bc[i] = t[i];
      ctl[0] = bad;
    }
    __syncthreads();
    for (int i = 0; i < 4; ++i) v[i] = bc[i];
    if (ctl[0]) fail = true;
    __syncthreads();
  }

  // ---- one sweep -----------------------------------------------------------
  template <typename T>
  __device__ void run_sweep(const Sweep<T>& sw, double acc[4]) {
    const int kind = sw.kind;
    const Geo gg = geo(kind);
    const int R = gg.R, k = gg.k;
    const int bse = (kind == kKA64) ? bs64 : bs;  // element stride of a block
    T* ring = reinterpret_cast<T*>(sm + kSmRing);
    T* vs = reinterpret_cast<T*>(sm + kSmVs);
    T* part1 = reinterpret_cast<T*>(sm + kSmParts);
    T* part2 = part1 + kMaxChunkElems;
    T* push = part2 + kMaxChunkElems;
    const int nc = (e - s + R - 1) / R;
    for (int c = 0; c < nc; ++c) {
      const int r0 = s + c * R;
      const int r1 = min(e, r0 + R);
      const int nr = r1 - r0;
      const int h = (c == 0) ? min(gg.halo, s) : 0;
      const int base = r0 - h;
      const int vend = min(N, r1 + k);
      const int st = consumed % S;
      const unsigned par = (consumed / S) & 1u;
      // 1. wait for the chunk's blocks (every thread observes the mbarrier)
      const bool ok = mbar_wait(&full[st], par, deadline + (1ll << 31));
      ++consumed;
      // 2. stage the vector rows [base, vend) with the fused PCG updates
      const int nv = (vend - base) * n;
      for (int t = tid; t < nv; t += kThreads) {
        const int row = base + t / n;
        const long long idx = (long long)row * n + (t % n);
        const bool own = row >= r0 && row < r1;
        T v;
        switch (sw.stg) {
          case SV_P: {
            v = sw.first ? sw.z[idx] : fma(sw.beta, sw.p_old[idx], sw.z[idx]);
            if (own) sw.p_cur[idx] = v;
          } break;
          case SV_VEC:
            v = static_cast<T>(sw.src64[idx]);
            break;
          case SV_R_UPD: {
            v = fma(-sw.alpha, sw.q[idx], sw.r_old[idx]);
            if (own) {
              sw.r_cur[idx] = v;
              sw.x[idx] = fma(sw.alpha, sw.p_in[idx], sw.x[idx]);
              acc[2] += (double)v * (double)v;
            }
          } break;
          case SV_R_FIRST: {
            v = static_cast<T>(sw.src64[idx] * sw.scale);
            if (own) {
              if (sw.write_r) sw.r_cur[idx] = v;
              if (sw.zero_x) sw.x[idx] = T(0);
              acc[2] += (double)v * (double)v;
            }
          } break;
          case SV_R_X0: {
            v = static_cast<T>(sw.src64[idx] - (double)sw.q[idx]);
            if (own) {
              sw.r_cur[idx] = v;
              acc[2] += (double)v * (double)v;
            }
          } break;
          default:
            v = sw.yprev[idx];
            break;
        }
        vs[t] = v;
      }
      if (__syncthreads_or(!ok)) {
        fail = true;
        if (G > 1 && tid == 0) atomicExch(P.abort_flag, 1);
        return;
      }
      // 3. block-vector products out of shared memory
      const T* stg = reinterpret_cast<const T*>(stages + (size_t)st * SB);
      const T* a0 = stg;
      const T* a1 = stg + (size_t)R * bse;
      const T* a2 = stg + (size_t)2 * R * bse;
      const int nd = nr * n;
      const int ntask = 2 * nd + (nr + h) * n;
      for (int t = tid; t < ntask; t += kThreads) {
        if (t < nd) {
          const int jj = t / n, a = t - jj * n;
          const int row = r0 + jj;
          part1[t] = dot_col(a0 + (size_t)jj * bse, n, a, vs + (row - base) * n);
        } else if (t < 2 * nd) {
          const int t2 = t - nd;
          const int jj = t2 / n, a = t2 - jj * n;
          const int row = r0 + jj;
          T val = T(0);
          if (row + k < N) {
            const T* M2 = (kind == kKB2) ? a1 + (size_t)jj * bse : a1 + (size_t)(jj + h) * bse;
            val = dot_col(M2, n, a, vs + (row + k - base) * n);
          }
          part2[t2] = val;
        } else {
          const int t3 = t - 2 * nd;
          const int jj = t3 / n, a = t3 - jj * n;
          const int src = base + jj;
          T val = T(0);
          if (src + k < N) {
            if (kind == kKB2) val = dot_col(a2 + (size_t)jj * bse, n, a, vs + jj * n);
            else val = dot_tr(a1 + (size_t)jj * bse, n, a, vs + jj * n);
          }
          push[t3] = val;
        }
      }
      __syncthreads();
      // 4. the stage is free: refill it with the next predicted chunk
      advance_producer_after_release();
      // 5. finalize owned rows
      for (int t = tid; t < nd; t += kThreads) {
        const int jj = t / n, a = t - jj * n;
        const int row = r0 + jj;
        const int src = row - k;
        T carry = T(0);
        if (src >= 0) carry = (src >= base) ? push[(src - base) * n + a] : ring[(src % k) * n + a];
        const T out = part1[t] + sw.sgn * (part2[t] + carry);
        const long long idx = (long long)row * n + a;
        const T vi = vs[(row - base) * n + a];
        switch (sw.fin) {
          case FN_Q:
            sw.qout[idx] = out;
            acc[0] += (double)vi * (double)out;
            break;
          case FN_OUT64:
            sw.out64[idx] = (double)out;
            break;
          case FN_R64: {
            const double r = sw.bsub[idx] - (double)out;
            sw.r64[idx] = r;
            acc[0] += r * r;
          } break;
          case FN_Y0:
            if (sw.m1) {
              if (sw.out_to_user) sw.out64[idx] = (double)out;
              else sw.zv[idx] = out;
              acc[1] += (double)vi * (double)out;
            } else {
              sw.y0[idx] = out;
            }
            break;
          default: {  // FN_YJ
            const T zprev = (sw.j == 1) ? vi : sw.zv[idx];
            const T zz = fma(sw.alpha_j, out, zprev);
            if (!sw.last) sw.ynext[idx] = out;
            if (sw.last && sw.out_to_user) sw.out64[idx] = (double)zz;
            else sw.zv[idx] = zz;
            if (sw.last) acc[1] += (double)sw.rcur_for_dot[idx] * (double)zz;
          } break;
        }
      }
      __syncthreads();
      // 6. keep the last k pushes for the next chunk
      for (int t = tid; t < k * n; t += kThreads) {
        const int w = t / n, a = t - w * n;
        const int src = r1 - k + w;
        if (src >= base && src >= 0) ring[(src % k) * n + a] = push[(src - base) * n + a];
      }
    }
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
template <typename MT>
__device__ void solve_instance(Solver<MT>& Sv, int inst_id);

template <typename MT>
__global__ void __launch_bounds__(kThreads, 2) bt_persistent_kernel(const __grid_constant__ KParams P) {
  extern __shared__ __align__(128) char smem[];
  Solver<MT> Sv(P, smem);
  if (threadIdx.x == 0) {
    for (int i = 0; i < P.stages; ++i) mbar_init(&Sv.full[i], 1);
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
    solve_instance<MT>(Sv, inst);
    if (P.G > 1) break;
  }
}

template <typename MT>
__device__ void solve_instance(Solver<MT>& Sv, int inst_id) {
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
  const int N = d.N, n = d.n, m = P.m;
  if (sizeof(MT) == 4) {
    const long long o = d.off32;
    Sv.mats[0] = (const MT*)(P.D32 + o); Sv.mats[1] = (const MT*)(P.O32 + o);
    Sv.mats[2] = (const MT*)(P.Dinv32 + o); Sv.mats[3] = (const MT*)(P.E32 + o);
    Sv.mats[4] = (const MT*)(P.Hd32 + o); Sv.mats[5] = (const MT*)(P.Hu32 + o);
    Sv.mats[6] = (const MT*)(P.Hl32 + o);
  } else {
    const long long o = d.off64;
    Sv.mats[0] = (const MT*)(P.D64 + o); Sv.mats[1] = (const MT*)(P.O64 + o);
    Sv.mats[2] = (const MT*)(P.Dinv64 + o); Sv.mats[3] = (const MT*)(P.E64 + o);
    Sv.mats[4] = (const MT*)(P.Hd64 + o); Sv.mats[5] = (const MT*)(P.Hu64 + o);
    Sv.mats[6] = (const MT*)(P.Hl64 + o);
  }
  Sv.mats64[0] = P.D64 + d.off64;
  Sv.mats64[1] = P.O64 + d.off64;

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
  int pat_it[kMaxM + 2];
  pat_it[0] = kKA;
  pat_it[1] = kKB1;
  for (int j = 1; j < m; ++j) pat_it[1 + j] = kKB2;
  const int pat_it_len = m + 1;

  double acc[4];
  auto zero_acc = [&]() { acc[0] = acc[1] = acc[2] = acc[3] = 0.0; };

  // Apply z = M^-1 rhs into the inner vectors (or to the user array).
  // Runs B1 then B2 x (m-1); rz accumulates in acc[1] of the last sweep.
  // rhs given by (src64, scale) when first_from_user, else r already staged
  // through SV_R_UPD by the caller.
  auto precond_sweeps_after_b1 = [&](MT* rcur, bool to_user) {
    for (int j = 1; j < m; ++j) {
      Sweep<MT> sw = {};
      sw.kind = kKB2; sw.stg = SV_Y; sw.fin = FN_YJ; sw.sgn = MT(1);
      sw.yprev = (j == 1) ? y0 : ((j - 1) % 2 == 1 ? ya : yb);
      sw.ynext = (j % 2 == 1) ? ya : yb;
      sw.zv = z; sw.j = j; sw.m = m; sw.alpha_j = (MT)P.alpha[j]; sw.last = (j == m - 1);
      sw.rcur_for_dot = rcur; sw.out_to_user = to_user; sw.out64 = xu;
      zero_acc();
      Sv.run_sweep(sw, acc);
      Sv.group_reduce(acc);
      if (Sv.fail) return;
    }
  };

  int iters_total = 0, outer = 0;
  double resid = 0.0, errv = 0.0;

  if (P.op == kOpSpmv64 || (P.op == kOpSpmv32 && sizeof(MT) == 8)) {
    const int pat[1] = {kKA64};
    Sv.restart(pat, 1, 0);
    Sweep<double> sw = {};
    sw.kind = kKA64; sw.stg = SV_VEC; sw.fin = FN_OUT64; sw.sgn = 1.0;
    sw.src64 = bu; sw.out64 = xu;
    zero_acc();
    Sv.run_sweep(sw, acc);
    Sv.group_reduce(acc);
  } else if (P.op == kOpSpmv32) {
    const int pat[1] = {kKA};
    Sv.restart(pat, 1, 0);
    Sweep<MT> sw = {};
    sw.kind = kKA; sw.stg = SV_VEC; sw.fin = FN_OUT64; sw.sgn = MT(1);
    sw.src64 = bu; sw.out64 = xu;
    zero_acc();
    Sv.run_sweep(sw, acc);
    Sv.group_reduce(acc);
  } else if (P.op == kOpApply) {
    Sv.restart(pat_it, pat_it_len, 1);
    Sweep<MT> sw = {};
    sw.kind = kKB1; sw.stg = SV_R_FIRST; sw.fin = FN_Y0; sw.sgn = MT(-1);
    sw.src64 = bu; sw.scale = 1.0; sw.r_cur = rb[0]; sw.write_r = true; sw.zero_x = false;
    sw.y0 = y0; sw.m1 = (m == 1); sw.out_to_user = true; sw.out64 = xu; sw.zv = z;
    zero_acc();
    Sv.run_sweep(sw, acc);
    Sv.group_reduce(acc);
    if (!Sv.fail) precond_sweeps_after_b1(rb[0], true);
  } else {
    // ------------------------------ SOLVE ------------------------------
    // Inner PCG on S d = rhs (rhs from src64 * scale or b - S x0), textbook
    // form; returns iterations, sets status, leaves the solution in xvec.
    auto inner_pcg = [&](const double* src64, double scale, MT* xv, bool from_x0, double tol_rel,
                         int maxit, int& it_out, int& st_out, double& rr_out) {
      it_out = 0;
      st_out = kOK;
      // initial residual and z0 = M^-1 r0
      Sv.restart(pat_it, pat_it_len, from_x0 ? 0 : 1);
      if (from_x0) {
        Sweep<MT> sa = {};
        sa.kind = kKA; sa.stg = SV_VEC; sa.fin = FN_Q; sa.sgn = MT(1);
        sa.src64 = reinterpret_cast<const double*>(xv);  // float64 path only
        sa.qout = q;
        zero_acc();
        Sv.run_sweep(sa, acc);
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
      Sv.run_sweep(s1, acc);
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
      if (sqrt(rr) <= tol_rel * nrhs) { return; }
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
        Sv.run_sweep(sa, acc);
        Sv.group_reduce(acc);
        if (Sv.fail || acc[3] > 0) { st_out = kErrTimeout; it_out = k - 1; return; }
        const double pq = acc[0];
        if (!isfinite(pq)) { st_out = kErrNonfinite; it_out = k - 1; return; }
        if (!(pq > 0.0)) { st_out = kErrBreakdown; it_out = k - 1; errv = pq; return; }
        const double alpha = rho / pq;
        // B1: r -= alpha q, x += alpha p, y0 = G r
        Sweep<MT> sb = {};
        sb.kind = kKB1; sb.stg = SV_R_UPD; sb.fin = FN_Y0; sb.sgn = MT(-1);
        sb.alpha = (MT)alpha; sb.r_old = rb[(k + 1) & 1]; sb.r_cur = rb[k & 1]; sb.q = q;
        sb.x = xv; sb.p_in = pb[k & 1];
        sb.y0 = y0; sb.m1 = (m == 1); sb.out_to_user = false; sb.zv = z;
        zero_acc();
        Sv.run_sweep(sb, acc);
        Sv.group_reduce(acc);
        if (Sv.fail || acc[3] > 0) { st_out = kErrTimeout; it_out = k; return; }
        rr = acc[2];
        rr_out = rr;
        it_out = k;
        if (!isfinite(rr)) { st_out = kErrNonfinite; return; }
        if (sqrt(rr) <= tol_rel * nrhs) return;
        if (m > 1) {
          precond_sweeps_after_b1(rb[k & 1], false);
          if (Sv.fail) { st_out = kErrTimeout; return; }
        }
        const double rz_new = acc[1];
        beta = rz_new / rho;
        rho = rz_new;
      }
    };

    if (!mixed) {
      // float64 path: PCG directly on the user vectors
      int it, st;
      double rr;
      MT* xv = reinterpret_cast<MT*>(xu);
      inner_pcg(bu, 1.0, xv, P.use_x0 != 0, P.tol, P.maxit, it, st, rr);
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
            const int pat[1] = {kKA64};
            Sv.restart(pat, 1, 0);
            Sweep<double> sw = {};
            sw.kind = kKA64; sw.stg = SV_VEC; sw.fin = FN_R64; sw.sgn = 1.0;
            sw.src64 = xu; sw.bsub = bu; sw.r64 = r64;
            zero_acc();
            Sv.run_sweep(sw, acc);
            Sv.group_reduce(acc);
            if (Sv.fail || acc[3] > 0) { st = kErrTimeout; break; }
            nr = sqrt(acc[0]);
            if (!isfinite(nr)) { st = kErrNonfinite; break; }
          }
          resid = nr / nb;
          if (nr <= tol * nb) { st = kOK; break; }
          if (outer >= P.max_outer || iters_total >= P.maxit) { st = kErrNoConv; break; }
          double t_in = P.tol_inner;
          const double need = 0.5 * tol * nb / nr;
          if (need > t_in) t_in = need;
          if (t_in > 0.5) t_in = 0.5;
          int it, ist;
          double rr;
          inner_pcg(have_r64 ? r64 : bu, 1.0 / nr, x_in, false, t_in, P.maxit - iters_total, it, ist, rr);
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

// Explicit instantiations and host launchers.
template __global__ void bt_persistent_kernel<float>(const __grid_constant__ KParams P);
template __global__ void bt_persistent_kernel<double>(const __grid_constant__ KParams P);

}  // namespace bt

// Host-side entry used by bt_api.cu.
extern "C" cudaError_t bt_launch_persistent(const bt::KParams* P, int grid, int smem_bytes, int mt_is_float,
                                            int cooperative, cudaStream_t stream) {
  const void* fn = mt_is_float ? (const void*)bt::bt_persistent_kernel<float>
                               : (const void*)bt::bt_persistent_kernel<double>;
  cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (err != cudaSuccess) return err;
  void* args[] = {(void*)P};
  if (cooperative) return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(bt::kThreads), args, smem_bytes, stream);
  return cudaLaunchKernel(fn, dim3(grid), dim3(bt::kThreads), args, smem_bytes, stream);
}

extern "C" int bt_persistent_smem_fixed() { return bt::smem_fixed_bytes(); }

extern "C" cudaError_t bt_persistent_occupancy(int mt_is_float, int smem_bytes, int* blocks_per_sm) {
  const void* fn = mt_is_float ? (const void*)bt::bt_persistent_kernel<float>
                               : (const void*)bt::bt_persistent_kernel<double>;
  cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (err != cudaSuccess) return err;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, bt::kThreads, smem_bytes);
}
