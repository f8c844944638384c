// C ABI of libbt (declared in include/bt.h): argument checks, memory layout,
// instance scheduling order, launch configuration and the entry points.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/bt.h"
#include "bt_alpha.h"
#include "bt_common.cuh"

extern "C" cudaError_t bt_launch_persistent(const bt::KParams* P, int grid, int smem_bytes, int mt_is_float,
                                            int cooperative, cudaStream_t stream);
extern "C" int bt_persistent_smem_fixed(int variant);
extern "C" cudaError_t bt_persistent_occupancy(int mt_is_float, int variant, int smem_bytes, int* blocks_per_sm);
extern "C" cudaError_t bt_launch_setup(const bt::SetupParams* P, int mixed, int m, int maxn, cudaStream_t st);
extern "C" bt_status bt_lqr_schur_handle(int B, const int* N, const int* n, const int* m, const double* A,
                                         const double* Bm, const double* Q, const double* R, const double* q,
                                         const double* r, const double* c, double* gamma, const bt::InstDesc* hinst,
                                         double* hD64, double* hO64, float* hD32, float* hO32, float* hDinv32,
                                         void* stream, int* bad_inst, int* bad_row, void* buf, size_t buf_bytes,
                                         size_t* need);
extern "C" size_t bt_lqr_handle_bytes(int B, const int* N, const int* n, const int* m);
extern "C" bt_status bt_lqr_recover_w_run(int B, const int* N, const int* n, const int* m, const double* A,
                                          const double* Bm, const double* q, const double* r, const double* lambda,
                                          double* x, double* u, const void* buf, void* stream);
extern "C" cudaError_t bt_launch_adjoint(const bt::AdjParams* P, cudaStream_t st);
namespace bt { struct MParams; }
extern "C" int bt_mrhs_smem_bytes(int n, int tc);
extern "C" int bt_small_cluster(int N, int n, int bs64, int bs32, int want);
extern "C" cudaError_t bt_small_launch(const double* const* blk64, const float* const* blk32, int N, int n, int bs64,
                                       int bs32, int m, const double* alpha, const double* b, double* x, int use_x0,
                                       double tol, double tol_inner, int max_outer, int maxit, long long budget,
                                       double* hist, int hist_len, int* iters, int* status, int* outer,
                                       double* resid, double* errval, int scal64, int C, cudaStream_t st);
extern "C" int bt_mrhs_tc_supported(int n);
extern "C" cudaError_t bt_mrhs_occupancy(int smem, int tc, int* blocks);
extern "C" cudaError_t bt_mrhs_images(int N, int n, int m, const float* const* blk32, int bs32, float* const* img,
                                      cudaStream_t st);
extern "C" cudaError_t bt_mrhs_solve_launch(int N, int n, int m, const double* alpha, const float* const* blk32,
                                            const double* D64, const double* O64, int bs32, int bs64,
                                            void* const* vec, const float* const* img, double tol, double tol_inner,
                                            int maxit, int max_outer, long long budget, int G, int nrhs,
                                            const double* B, double* X, int smem, cudaStream_t st);

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct bt_ctx {
  bool batched = false;
  int B = 0;
  std::vector<int> N, n;
  std::vector<long long> d_off, o_off, vec_off;
  int maxN = 0, maxn = 0;
  long long maxNn = 0, total_rows = 0, total_vec = 0;
  bt_params prm{};
  double alpha[BT_MAX_M];
  cudaStream_t stream = nullptr;
  int mixed = 0;
  int dev = 0, sms = 0;
  // device memory
  std::vector<void*> allocs;
  size_t bytes = 0;
  double *D64 = nullptr, *O64 = nullptr, *Dinv64 = nullptr, *E64 = nullptr, *Hd64 = nullptr, *Hu64 = nullptr,
         *Hl64 = nullptr;
  float *D32 = nullptr, *O32 = nullptr, *Dinv32 = nullptr, *E32 = nullptr, *Hd32 = nullptr, *Hu32 = nullptr,
        *Hl32 = nullptr;
  // general member of the family (a < 1, m >= 2): the +-1 blocks of H_ab
  double *F64 = nullptr, *K64 = nullptr;
  float *F32 = nullptr, *K32 = nullptr;
  int variant = 0;  // persistent kernel: 0 stored H_opt, 1 general member, 2 matrix-free H_opt
  int small = 0;    // single float64 instance on the shared-memory engine (bt_small.cu): its cluster size, 0 = off
  double* hist = nullptr;  // caller's per-iteration history buffer (bt_set_history), or null
  int hist_len = 0;
  bt::InstDesc* d_inst = nullptr;
  bt::RowRef* d_rows = nullptr;
  int* d_order = nullptr;
  long long* d_doff = nullptr;
  long long* d_ooff = nullptr;
  int* d_ctl = nullptr;          // [0] queue, [1] abort, [2] barrier (as unsigned)
  double* d_red = nullptr;
  int *d_iters = nullptr, *d_status = nullptr, *d_outer = nullptr;
  double *d_resid = nullptr, *d_errval = nullptr;
  unsigned long long* d_fail_key = nullptr;
  double* d_fail_piv = nullptr;
  int* d_retry = nullptr;  // mixed: float64 refactor list (count + rows)
  bt::SegRef* d_segs = nullptr;  // mixed: row segments of the fused E/H kernel
  long long nsegs = 0;
  long long* d_cls_idx = nullptr;  // mixed: canonical rows grouped by block-size class (float32 factor)
  long long cls_lo[4] = {}, cls_hi[4] = {};
  long long seg_lo[4] = {}, seg_hi[4] = {};  // mixed: the E/H segments of each class (grouped in d_segs)
  char* d_ws = nullptr;
  long long ws_stride = 0, ws_vec = 0;
  int ws_slots = 0;
  int ws_cap = 0;  // workspace slots allocated (a later configure() may not exceed them)
  // launch configuration
  int stages = 0, stage_bytes = 0, smem = 0, grid = 0, G = 1, vec_slot_bytes = 0;
  // results of the last solve
  std::vector<int> h_outer;
  std::vector<double> h_resid;
  // last error detail
  int err_inst = -1, err_blk = -1;
  double err_val = 0.0;
  cudaGraphExec_t graph = nullptr;
  cudaGraph_t graph_src = nullptr;
  // many-right-hand-side workspace (allocated on the first bt_pcg_solve_multi)
  void* mr_vec[17] = {};
  int mr_G = 0, mr_smem = 0, mr_outer = 0;
  float* mr_img[9] = {};  // block images of the tensor-core many-RHS engine
  void* lqr_buf = nullptr;  // bt_lqr_refactor's scratch (kept after its first call): the W factors
  size_t lqr_bytes = 0;
  bool lqr_valid = false;   // the W factors belong to the last bt_lqr_refactor
  std::vector<int> lqr_m;   // its input sizes
  std::vector<double> mr_resid;
};

namespace bt {
// One power-iteration step per instance (one CTA each): hv = v - u with
// u = G (S v), then v <- hv / ||hv|| and est = ||hv||.  first: v <- the fixed
// start vector 1 + sin(i)/10 (i the element index in the instance), normalised.
__global__ void k_rho_step(const InstDesc* inst, double* v, const double* u, double* est, int first) {
  __shared__ double red[32];
  const InstDesc d = inst[blockIdx.x];
  const long long len = (long long)d.N * d.n;
  double* vv = v + d.vec;
  const double* uu = u + d.vec;
  double s = 0.0;
  for (long long t = threadIdx.x; t < len; t += blockDim.x) {
    const double h = first ? 1.0 + 0.1 * sin((double)t) : vv[t] - uu[t];
    vv[t] = h;
    s += h * h;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    red[0] = sqrt(t);
  }
  __syncthreads();
  const double nrm = red[0];
  const double sc = nrm > 0.0 ? 1.0 / nrm : 0.0;
  for (long long t = threadIdx.x; t < len; t += blockDim.x) vv[t] *= sc;
  if (threadIdx.x == 0 && !first) est[blockIdx.x] = nrm;
}
}  // namespace bt

namespace {

inline bt_status cuda_st(cudaError_t e) { return e == cudaSuccess ? BT_OK : BT_ERR_CUDA; }

// NVTX range over an entry point (host-side span of the call; the kernels it
// queues show up inside it on a profiler's timeline).  Header-only NVTX: no
// cost unless a tool is attached.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

template <typename T>
bt_status dalloc(bt_ctx* h, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  void* q = nullptr;
  if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) return BT_ERR_ALLOC;
  h->allocs.push_back(q);
  h->bytes += count * sizeof(T);
  *p = static_cast<T*>(q);
  return BT_OK;
}

void free_all(bt_ctx* h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  if (h->graph_src) cudaGraphDestroy(h->graph_src);
  h->graph = nullptr;
  h->graph_src = nullptr;
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
  if (h->lqr_buf) cudaFree(h->lqr_buf);
  h->lqr_buf = nullptr;
  h->lqr_bytes = 0;
}

bt_status check_params(const bt_params* p, double* alpha_out) {
  if (!p) return BT_ERR_ARG;
  // admissible set C_g (Sec. 3.3): a in [0, 1], b = 1 - 2a
  if (!(p->a >= 0.0 && p->a <= 1.0)) return BT_ERR_PARAM;
  if (p->m < 1 || p->m > BT_MAX_M) return BT_ERR_PARAM;
  for (int j = 0; j < p->m; ++j) {
    const double a = p->alpha ? p->alpha[j] : 1.0;
    if (!std::isfinite(a)) return BT_ERR_PARAM;
    alpha_out[j] = a;
  }
  if (alpha_out[0] != 1.0) return BT_ERR_PARAM;
  // M^-1 SPD for every admissible S: q(h) = sum alpha_j h^j > 0 on [0, 1]
  if (!bt::alpha_positive_on_unit_interval(alpha_out, p->m)) return BT_ERR_PARAM;
  // polynomial coefficients belong to (G_opt, H_opt) (Sec. 3.5, Thm. 3.3): H_opt
  // has eigenvalues in [0, 1), so alpha_j >= 0 keeps M^-1 SPD; H_ab of a < 1 has
  // negative eigenvalues too, where such a polynomial can turn M^-1 indefinite
  if (p->a != 1.0)
    for (int j = 0; j < p->m; ++j)
      if (alpha_out[j] != 1.0) return BT_ERR_PARAM;
  if (p->precision != BT_FP64 && p->precision != BT_MIXED) return BT_ERR_PARAM;
  if (p->tol_inner < 0.0 || p->tol_inner >= 1.0) return BT_ERR_PARAM;
  if (p->max_outer < 0 || p->cycle_budget < 0 || p->ctas_per_sm < 0 || p->group_ctas < -8 || p->stage_kb < 0)
    return BT_ERR_PARAM;
  // the matrix-free H applies H_opt = H_J^2: the optimum only
  if (p->h_matrix_free != 0 && (p->h_matrix_free != 1 || p->a != 1.0)) return BT_ERR_PARAM;
  if (p->mrhs_engine < 0 || p->mrhs_engine > 2) return BT_ERR_PARAM;
  if (p->mixed_strict_fp64 != 0 && p->mixed_strict_fp64 != 1) return BT_ERR_PARAM;
  return BT_OK;
}

inline long long rup(long long v, long long a) { return (v + a - 1) / a * a; }

// The block-size classes of the float32 factor (mixed handles), or none.
void set_classes(const bt_ctx* h, bt::SetupParams& sp) {
  sp.cls_idx = h->d_cls_idx;
  for (int c = 0; c < 4; ++c) {
    sp.cls_lo[c] = h->cls_lo[c];
    sp.cls_hi[c] = h->cls_hi[c];
    sp.seg_lo[c] = h->seg_lo[c];
    sp.seg_hi[c] = h->seg_hi[c];
  }
}

// Queue the setup kernels (K0..K3) for D, O on the handle's stream.
bt_status launch_setup_kernels(bt_ctx* h, const double* D, const double* O) {
  cudaStream_t st = h->stream;
  if (cudaMemsetAsync(h->d_fail_key, 0xff, sizeof(unsigned long long), st)) return BT_ERR_CUDA;
  bt::SetupParams sp{};
  sp.inst = h->d_inst;
  sp.rows = h->d_rows;
  sp.nrows = h->total_rows;
  sp.D = D;
  sp.O = O;
  sp.d_off = h->d_doff;
  sp.o_off = h->d_ooff;
  sp.D64 = h->D64; sp.O64 = h->O64; sp.Dinv64 = h->Dinv64; sp.E64 = h->E64;
  sp.Hd64 = h->Hd64; sp.Hu64 = h->Hu64; sp.Hl64 = h->Hl64;
  sp.D32 = h->D32; sp.O32 = h->O32; sp.Dinv32 = h->Dinv32; sp.E32 = h->E32;
  sp.Hd32 = h->Hd32; sp.Hu32 = h->Hu32; sp.Hl32 = h->Hl32;
  sp.F64 = h->F64; sp.K64 = h->K64; sp.F32 = h->F32; sp.K32 = h->K32;
  sp.fam_a = h->prm.a;
  sp.want32 = h->mixed ? 1 : 0;
  sp.want64 = 1;
  sp.fail_key = h->d_fail_key;
  sp.fail_piv = h->d_fail_piv;
  // the strict float64 split factors every D_i in float64 (no float32 factor to refuse)
  sp.retry = h->prm.mixed_strict_fp64 ? nullptr : h->d_retry;
  sp.segs = h->d_segs;
  sp.nsegs = h->nsegs;
  set_classes(h, sp);
  // the matrix-free variant forms no H blocks
  return cuda_st(bt_launch_setup(&sp, h->mixed ? 1 : 0, h->variant == 2 ? 1 : h->prm.m, h->maxn, st));
}

// Read the setup failure key (synchronises); fills the error detail.
bt_status read_setup_status(bt_ctx* h) {
  unsigned long long key = 0;
  if (cudaMemcpyAsync(&key, h->d_fail_key, sizeof(key), cudaMemcpyDeviceToHost, h->stream)) return BT_ERR_CUDA;
  if (cudaStreamSynchronize(h->stream)) return BT_ERR_CUDA;
  if (key == ~0ull) return BT_OK;
  h->err_inst = (int)(key >> 32);
  h->err_blk = (int)(key & 0xffffffffu);
  long long grow = 0;
  for (int k = 0; k < h->err_inst; ++k) grow += h->N[k];
  grow += h->err_blk;
  cudaMemcpy(&h->err_val, h->d_fail_piv + grow, sizeof(double), cudaMemcpyDeviceToHost);
  return BT_ERR_NOT_SPD;
}

// Launch shape of the persistent kernel for a stage size and (single
// instance) a CTA count; 0 = the defaults.  Sets stages, stage and vector-slot
// bytes, dynamic shared memory, grid and group size; allocates nothing.
// The cluster size of the shared-memory engine for a single-instance handle
// (the optimum with stored H blocks, float64 or mixed): `want` CTAs (want >
// 0), or the smallest cluster whose CTAs hold the blocks (want = 0); 0 where
// none does.
int small_cluster(const bt_ctx* h, int want) {
  if (h->batched || h->variant != 0 || h->B != 1) return 0;
  const int n = h->n[0];
  return bt_small_cluster(h->N[0], n, (int)rup((long long)n * n, 2), h->mixed ? bt::slot32(n) : 0, want);
}

bt_status configure(bt_ctx* h, int stage_kb, int group_ctas) {
  // single instances: group_ctas -C asks for the shared-memory engine on a
  // cluster of C CTAs, 0 takes it (smallest cluster) where eligible; the
  // persistent kernel's shape is configured either way
  if (group_ctas < 0 && group_ctas != -1 && group_ctas != -2 && group_ctas != -4 && group_ctas != -8)
    return BT_ERR_ARG;
  h->small = group_ctas <= 0 ? small_cluster(h, -group_ctas) : 0;
  if (group_ctas < 0 && !h->small) return BT_ERR_ARG;
  if (group_ctas < 0) group_ctas = 0;
  const bool mixed = h->mixed != 0;
  const bool general = h->variant == 1;
  const bool mf = h->variant == 2;
  const int B = h->B;
  const int wbytes = mixed ? 4 : 8;
  long long bsb_max = rup((long long)h->maxn * h->maxn, 2) * wbytes;
  if (mixed)
    for (int q = 1; q <= h->maxn; ++q) bsb_max = std::max<long long>(bsb_max, (long long)bt::slot32(q) * wbytes);
  const long long bsb64_max = rup((long long)h->maxn * h->maxn, 2) * 8;
  // one chunk of one row: 3 + 2 halo blocks for H, 5 + 4 for H_ab, 3 float64
  long long need = std::max((general ? 9 : (mf ? 3 : 5)) * bsb_max, 3 * bsb64_max);
  long long sb = stage_kb > 0 ? (long long)stage_kb * 1024 : 80 * 1024;
  sb = std::max(sb, rup(need, 128));
  int smem_optin = 0;
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->dev);
  const int fixed = bt_persistent_smem_fixed(h->variant);
  int vslot = mixed ? 9 * 1024 : 18 * 1024;  // one vector-ring slot (largest chunk plan)
  int cps = h->prm.ctas_per_sm > 0 ? h->prm.ctas_per_sm : 1;
  const int per_cta = (int)std::min<long long>(smem_optin, (228 * 1024) / cps - 1024);
  const int vslots = (h->variant) == 1 ? 3 : 4;  // vector ring slots of the kernel variant
  int S = (int)((per_cta - fixed - vslots * vslot) / sb);
  if (S < 2) {  // large blocks: keep two block stages, stage vectors directly
    vslot = 0;
    S = (int)((per_cta - fixed) / sb);
  }
  h->vec_slot_bytes = vslot;
  if (S > bt::kMaxStages) S = bt::kMaxStages;
  if (S < 2) return BT_ERR_ARG;  // block too large for the shared-memory pipeline
  h->stages = S;
  h->stage_bytes = (int)sb;
  h->smem = fixed + vslots * vslot + S * (int)sb;
  int occ = 0;
  if (cuda_st(bt_persistent_occupancy(mixed ? 1 : 0, h->variant, h->smem, &occ)) != BT_OK || occ < 1)
    return BT_ERR_CUDA;
  cps = std::min(cps, occ);
  if (h->batched) {
    h->G = 1;
    h->grid = std::min(h->sms * cps, std::max(1, B));
    if (h->ws_cap > 0) h->grid = std::min(h->grid, h->ws_cap);
    h->ws_slots = h->grid;
  } else {
    int G = group_ctas;
    if (G <= 0) {
      // 4 block rows per CTA; one CTA up to N = 32, where the cross-CTA
      // reductions (3 per iteration) cost more than the rows they split
      // (LL^T N = 16, n = 6: 21.6 us per iteration on 1 CTA, 37.7 on 4)
      const int rows_per = 4;
      G = h->N[0] <= 32 ? 1 : std::max(1, std::min(h->sms * cps, h->N[0] / rows_per));
    }
    G = std::min(G, h->sms * std::min(occ, 2));
    G = std::min(G, h->N[0]);
    h->G = std::max(1, G);
    h->grid = h->G;
    h->ws_slots = 1;
  }
  return BT_OK;
}

// Common setup for one or many instances.
bt_status setup_common(bt_ctx* h, const double* D, const double* O) {
  cudaStream_t st = h->stream;
  cudaGetDevice(&h->dev);
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->dev);
  const int B = h->B;
  std::vector<bt::InstDesc> inst(B);
  long long off32 = 0, off64 = 0, vec = 0, rows = 0;
  for (int k = 0; k < B; ++k) {
    const int N = h->N[k], n = h->n[k];
    inst[k].N = N;
    inst[k].n = n;
    inst[k].bs32 = bt::slot32(n);
    inst[k].bs64 = (int)rup((long long)n * n, 2);
    inst[k].off32 = off32;
    inst[k].off64 = off64;
    inst[k].vec = vec;  // natural packing: instances back to back
    h->vec_off.push_back(vec);
    off32 += (long long)N * inst[k].bs32;
    off64 += (long long)N * inst[k].bs64;
    vec += (long long)N * n;
    rows += N;
    h->maxN = std::max(h->maxN, N);
    h->maxn = std::max(h->maxn, n);
    h->maxNn = std::max(h->maxNn, (long long)N * n);
  }
  h->total_rows = rows;
  h->total_vec = vec;
  const bool mixed = h->mixed != 0;
  const bool mf = h->prm.m >= 2 && h->prm.h_matrix_free == 1;  // H_opt = H_J^2 from D^-1, O
  const bool wantH = h->prm.m >= 2 && !mf;
  const bool general = wantH && h->prm.a != 1.0;  // H_ab has +-1 blocks
  h->variant = general ? 1 : (mf ? 2 : 0);
  bt_status s;
#define ALLOC(ptr, cnt) \
  if ((s = dalloc(h, &(ptr), (cnt))) != BT_OK) return s
  ALLOC(h->D64, off64);
  ALLOC(h->O64, off64);
  if (mixed) {
    ALLOC(h->D32, off32);
    ALLOC(h->O32, off32);
    ALLOC(h->Dinv32, off32);
    ALLOC(h->E32, off32);
    if (wantH) {
      ALLOC(h->Hd32, off32);
      ALLOC(h->Hu32, off32);
      ALLOC(h->Hl32, off32);
    }
    if (general) {
      ALLOC(h->F32, off32);
      ALLOC(h->K32, off32);
    }
  } else {
    ALLOC(h->Dinv64, off64);
    ALLOC(h->E64, off64);
    if (wantH) {
      ALLOC(h->Hd64, off64);
      ALLOC(h->Hu64, off64);
      ALLOC(h->Hl64, off64);
    }
    if (general) {
      ALLOC(h->F64, off64);
      ALLOC(h->K64, off64);
    }
  }
  ALLOC(h->d_inst, B);
  ALLOC(h->d_rows, rows);
  constexpr int kSegRows = 32;  // block rows per fused E/H segment
  if (mixed) {
    h->nsegs = 0;
    for (int k = 0; k < B; ++k) h->nsegs += (h->N[k] + kSegRows - 1) / kSegRows;
    ALLOC(h->d_segs, h->nsegs);
  }
  ALLOC(h->d_order, B);
  ALLOC(h->d_doff, B);
  ALLOC(h->d_ooff, B);
  ALLOC(h->d_ctl, 64);
  ALLOC(h->d_iters, B);
  ALLOC(h->d_status, B);
  ALLOC(h->d_outer, B);
  ALLOC(h->d_resid, B);
  ALLOC(h->d_errval, B);
  ALLOC(h->d_fail_key, 1);
  ALLOC(h->d_fail_piv, rows);
  if (h->mixed) {
    ALLOC(h->d_retry, rows + 1);
    ALLOC(h->d_cls_idx, rows);
  }
  // zero every block array once (padding slots must read as zero)
  auto z64 = [&](double* p) { if (p) cudaMemsetAsync(p, 0, off64 * sizeof(double), st); };
  auto z32 = [&](float* p) { if (p) cudaMemsetAsync(p, 0, off32 * sizeof(float), st); };
  z64(h->D64); z64(h->O64); z64(h->Dinv64); z64(h->E64); z64(h->Hd64); z64(h->Hu64); z64(h->Hl64);
  z32(h->D32); z32(h->O32); z32(h->Dinv32); z32(h->E32); z32(h->Hd32); z32(h->Hu32); z32(h->Hl32);
  z64(h->F64); z64(h->K64); z32(h->F32); z32(h->K32);
  // row table and LPT order (largest N n^2 first)
  std::vector<bt::RowRef> rr(rows);
  {
    long long t = 0;
    for (int k = 0; k < B; ++k)
      for (int i = 0; i < h->N[k]; ++i) rr[t++] = bt::RowRef{k, i};
  }
  // mixed: the rows of each block-size class of the float32 factor
  // (n = 12, 24, 36, other), canonical indices in instance order
  std::vector<long long> cls_idx;
  if (mixed) {
    cls_idx.reserve(rows);
    const auto cls_of = [](int n) { return n == 12 ? 0 : (n == 24 ? 1 : (n == 36 ? 2 : 3)); };
    for (int c = 0; c < 4; ++c) {
      h->cls_lo[c] = (long long)cls_idx.size();
      long long t = 0;
      for (int k = 0; k < B; ++k) {
        if (cls_of(h->n[k]) == c)
          for (int i = 0; i < h->N[k]; ++i) cls_idx.push_back(t + i);
        t += h->N[k];
      }
      h->cls_hi[c] = (long long)cls_idx.size();
    }
  }
  std::vector<bt::SegRef> segs;
  if (mixed) {  // grouped by block-size class, instance order within a class
    segs.reserve(h->nsegs);
    const auto cls_of = [](int n) { return n == 12 ? 0 : (n == 24 ? 1 : (n == 36 ? 2 : 3)); };
    for (int c = 0; c < 4; ++c) {
      h->seg_lo[c] = (long long)segs.size();
      for (int k = 0; k < B; ++k)
        if (cls_of(h->n[k]) == c)
          for (int a = 0; a < h->N[k]; a += kSegRows)
            segs.push_back(bt::SegRef{k, a, std::min(h->N[k], a + kSegRows), 0});
      h->seg_hi[c] = (long long)segs.size();
    }
  }
  std::vector<int> order(B);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (long long)h->N[a] * h->n[a] * h->n[a] > (long long)h->N[b] * h->n[b] * h->n[b];
  });
  const auto ok = [](cudaError_t x) { return x == cudaSuccess; };
  if (!ok(cudaMemcpyAsync(h->d_inst, inst.data(), B * sizeof(bt::InstDesc), cudaMemcpyHostToDevice, st)) ||
      !ok(cudaMemcpyAsync(h->d_rows, rr.data(), rows * sizeof(bt::RowRef), cudaMemcpyHostToDevice, st)) ||
      !ok(cudaMemcpyAsync(h->d_order, order.data(), B * sizeof(int), cudaMemcpyHostToDevice, st)) ||
      !ok(cudaMemcpyAsync(h->d_doff, h->d_off.data(), B * sizeof(long long), cudaMemcpyHostToDevice, st)) ||
      !ok(cudaMemcpyAsync(h->d_ooff, h->o_off.data(), B * sizeof(long long), cudaMemcpyHostToDevice, st)) ||
      (mixed && !ok(cudaMemcpyAsync(h->d_segs, segs.data(), segs.size() * sizeof(bt::SegRef),
                                     cudaMemcpyHostToDevice, st))) ||
      (mixed && !ok(cudaMemcpyAsync(h->d_cls_idx, cls_idx.data(), cls_idx.size() * sizeof(long long),
                                     cudaMemcpyHostToDevice, st))))
    return BT_ERR_CUDA;
  if (launch_setup_kernels(h, D, O) != BT_OK) return BT_ERR_CUDA;

  // ---- launch configuration of the persistent kernel ----
  if ((s = configure(h, h->prm.stage_kb, h->prm.group_ctas)) != BT_OK) return s;
  h->ws_vec = rup(std::max<long long>(h->maxNn, 1), 64);
  const int mts = mixed ? 4 : 8;
  h->ws_stride = rup(10 * h->ws_vec * mts + h->ws_vec * 8, 256);
  if ((s = dalloc(h, &h->d_ws, (size_t)h->ws_stride * h->ws_slots)) != BT_OK) return s;
  h->ws_cap = h->ws_slots;
  // group reduction slots for the largest group a later bt_autotune may choose
  if ((s = dalloc(h, &h->d_red, (size_t)2 * std::max(std::max(1, h->G), h->sms * 2) * 4)) != BT_OK) return s;
  cudaMemsetAsync(h->d_ws, 0, (size_t)h->ws_stride * h->ws_slots, st);

  // ---- setup status ----
  h->h_outer.assign(B, 0);
  h->h_resid.assign(B, 0.0);
  return read_setup_status(h);
}

bt_ctx* new_ctx(const bt_params* p) {
  bt_ctx* h = new bt_ctx();
  h->prm = *p;
  h->stream = static_cast<cudaStream_t>(p->stream);
  h->mixed = p->precision == BT_MIXED;
  return h;
}

bt::KParams base_kparams(bt_ctx* h) {
  bt::KParams P{};
  P.D64 = h->D64; P.O64 = h->O64; P.Dinv64 = h->Dinv64; P.E64 = h->E64;
  P.Hd64 = h->Hd64; P.Hu64 = h->Hu64; P.Hl64 = h->Hl64;
  P.D32 = h->D32; P.O32 = h->O32; P.Dinv32 = h->Dinv32; P.E32 = h->E32;
  P.Hd32 = h->Hd32; P.Hu32 = h->Hu32; P.Hl32 = h->Hl32;
  P.F64 = h->F64; P.K64 = h->K64; P.F32 = h->F32; P.K32 = h->K32;
  P.variant = h->variant;
  P.hist = h->hist;
  P.hist_len = h->hist_len;
  P.inst = h->d_inst;
  P.order = h->d_order;
  P.B = h->B;
  P.queue = h->d_ctl;
  P.abort_flag = h->d_ctl + 1;
  P.bar = reinterpret_cast<unsigned*>(h->d_ctl + 2);
  P.red = h->d_red;
  P.mixed = h->mixed;
  P.scal64 = h->prm.mixed_strict_fp64;
  P.m = h->prm.m;
  for (int j = 0; j < BT_MAX_M; ++j) P.alpha[j] = j < h->prm.m ? h->alpha[j] : 0.0;
  P.tol_inner = h->prm.tol_inner;  // 0: the kernel derives it from tol
  P.max_outer = h->prm.max_outer > 0 ? h->prm.max_outer : 30;
  P.use_x0 = h->prm.use_x0;
  P.budget = h->prm.cycle_budget > 0 ? h->prm.cycle_budget : (1ll << 34);
  P.ws = h->d_ws;
  P.ws_stride = h->ws_stride;
  P.ws_vec = h->ws_vec;
  P.G = h->G;
  P.iters = h->d_iters;
  P.status = h->d_status;
  P.outer = h->d_outer;
  P.resid = h->d_resid;
  P.errval = h->d_errval;
  P.stages = h->stages;
  P.stage_bytes = h->stage_bytes;
  P.vec_slot_bytes = h->vec_slot_bytes;
  return P;
}

bt_status launch(bt_ctx* h, bt::KParams& P) {
  cudaError_t e = cudaMemsetAsync(h->d_ctl, 0, 64 * sizeof(int), h->stream);
  if (e) return BT_ERR_CUDA;
  const bool coop = h->G > 1;
  e = bt_launch_persistent(&P, h->grid, h->smem, h->mixed, coop ? 1 : 0, h->stream);
  return cuda_st(e);
}

// Op launch with the batched grid or the group grid as configured.
bt_status run_op(bt_ctx* h, int op, const double* in, double* out) {
  bt::KParams P = base_kparams(h);
  P.op = op;
  P.bvec = in;
  P.xvec = out;
  P.tol = 0;
  P.maxit = 0;
  return launch(h, P);
}

bt_status collect(bt_ctx* h, int* iters, int* status_out, bool all) {
  const int B = h->B;
  std::vector<int> st(B), it(B);
  const auto ok = [](cudaError_t x) { return x == cudaSuccess; };
  if (!ok(cudaMemcpyAsync(it.data(), h->d_iters, B * sizeof(int), cudaMemcpyDeviceToHost, h->stream)) ||
      !ok(cudaMemcpyAsync(st.data(), h->d_status, B * sizeof(int), cudaMemcpyDeviceToHost, h->stream)) ||
      !ok(cudaMemcpyAsync(h->h_outer.data(), h->d_outer, B * sizeof(int), cudaMemcpyDeviceToHost, h->stream)) ||
      !ok(cudaMemcpyAsync(h->h_resid.data(), h->d_resid, B * sizeof(double), cudaMemcpyDeviceToHost,
                           h->stream)) ||
      !ok(cudaStreamSynchronize(h->stream)))
    return BT_ERR_CUDA;
  bt_status first = BT_OK;
  for (int k = 0; k < B; ++k) {
    if (iters) iters[k] = it[k];
    if (status_out) status_out[k] = st[k];
    if (st[k] != BT_OK && first == BT_OK) {
      first = static_cast<bt_status>(st[k]);
      h->err_inst = k;
      h->err_blk = -1;
      double v = 0;
      cudaMemcpy(&v, h->d_errval + k, sizeof(double), cudaMemcpyDeviceToHost);
      h->err_val = v;
    }
    if (!all) break;
  }
  return first;
}

}  // namespace

extern "C" {

// Key of a handle's shape in the tuning cache (BT_TUNE_CACHE).
static std::string tune_key(const bt_ctx* h) {
  long long sumN = 0;
  for (int v : h->N) sumN += v;
  char buf[256];
  std::snprintf(buf, sizeof(buf), "%s-v%d-p%d-m%d-B%d-N%lld-maxN%d-maxn%d-sms%d", h->batched ? "batched" : "single",
                h->variant, h->mixed, h->prm.m, h->B, sumN, h->maxN, h->maxn, h->sms);
  return buf;
}

bt_status bt_autotune(bt_handle h, const double* b, double* x, double tol, int maxit, int trials, int* stage_kb,
                      int* group_ctas) {
  Range nvtx_range("bt_autotune");
  if (!h || !b || !x || trials < 1 || !(tol >= 0.0) || maxit < 0) return BT_ERR_ARG;
  cudaStream_t st = h->stream;
  // tuning cache: one JSON object per line, {"key": "...", "stage_kb": K, "group_ctas": G}
  const char* cache = std::getenv("BT_TUNE_CACHE");
  const std::string key = tune_key(h);
  if (cache && *cache) {
    if (FILE* f = std::fopen(cache, "r")) {
      char line[512];
      int hit_kb = -1, hit_g = -1;
      while (std::fgets(line, sizeof(line), f)) {
        char k[300];
        int kb = 0, g = 0;
        if (std::sscanf(line, " {\"key\": \"%299[^\"]\", \"stage_kb\": %d, \"group_ctas\": %d", k, &kb, &g) == 3 &&
            key == k) {
          hit_kb = kb;
          hit_g = g;
        }
      }
      std::fclose(f);
      if (hit_kb >= 0 && configure(h, hit_kb, h->batched ? 0 : hit_g) == BT_OK) {
        if (h->graph) cudaGraphExecDestroy(h->graph);
        if (h->graph_src) cudaGraphDestroy(h->graph_src);
        h->graph = nullptr;
        h->graph_src = nullptr;
        h->prm.stage_kb = hit_kb;
        h->prm.group_ctas = h->batched ? 0 : (h->small ? -h->small : h->G);
        if (stage_kb) *stage_kb = h->stage_bytes / 1024;
        if (group_ctas) *group_ctas = h->small ? -h->small : h->G;
        const bt_status o = h->batched ? bt_pcg_solve_batched_async(h, b, x, tol, maxit, nullptr, nullptr)
                                       : bt_pcg_solve_async(h, b, x, tol, maxit, nullptr, nullptr);
        if (o != BT_OK) return o;
        return cudaStreamSynchronize(st) == cudaSuccess ? BT_OK : BT_ERR_CUDA;
      }
    }
  }
  // candidates: stage sizes for batched handles; for single instances the
  // shared-memory engine (group -1, where it fits) and CTAs per instance
  std::vector<std::pair<int, int>> cand;
  if (h->batched) {
    for (int kb : {64, 72, 80}) cand.push_back({kb, 0});
  } else {
    for (int C = 1; C <= 8; C *= 2)
      if (small_cluster(h, C)) cand.push_back({h->prm.stage_kb, -C});
    const int N = h->N[0];
    std::vector<int> gs = {1, N / 16, N / 8, N / 4, N / 2};
    for (int g : gs)
      if (g >= 1 && g <= N) {
        bool dup = false;
        for (auto& c : cand) dup = dup || c.second == g;
        if (!dup) cand.push_back({h->prm.stage_kb, g});
      }
  }
  if (h->graph) cudaGraphExecDestroy(h->graph);  // a captured graph holds the old shape
  if (h->graph_src) cudaGraphDestroy(h->graph_src);
  h->graph = nullptr;
  h->graph_src = nullptr;
  const int use_x0 = h->prm.use_x0;  // every timed solve starts from x = 0
  h->prm.use_x0 = 0;
  struct Restore {
    bt_ctx* h;
    int v;
    ~Restore() { h->prm.use_x0 = v; }
  } restore{h, use_x0};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return BT_ERR_CUDA;
  const auto solve = [&]() -> bt_status {
    return h->batched ? bt_pcg_solve_batched_async(h, b, x, tol, maxit, nullptr, nullptr)
                      : bt_pcg_solve_async(h, b, x, tol, maxit, nullptr, nullptr);
  };
  float best_ms = 0.f;
  int best = -1;
  bt_status out = BT_OK;
  for (size_t i = 0; i < cand.size() && out == BT_OK; ++i) {
    if (configure(h, cand[i].first, cand[i].second) != BT_OK) continue;  // shape does not fit: skip
    if ((out = solve()) != BT_OK) break;                                  // untimed
    cudaEventRecord(e0, st);
    for (int t = 0; t < trials && out == BT_OK; ++t) out = solve();
    cudaEventRecord(e1, st);
    if (out != BT_OK || cudaEventSynchronize(e1) != cudaSuccess) { out = out != BT_OK ? out : BT_ERR_CUDA; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (best < 0 || ms < best_ms) { best_ms = ms; best = (int)i; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best < 0) {
    configure(h, h->prm.stage_kb, h->prm.group_ctas);
    return out != BT_OK ? out : BT_ERR_ARG;
  }
  const bt_status cs = configure(h, cand[best].first, cand[best].second);
  if (cs != BT_OK) return cs;
  h->prm.stage_kb = cand[best].first;
  h->prm.group_ctas = h->batched ? 0 : (h->small ? -h->small : h->G);
  if (cache && *cache) {
    if (FILE* f = std::fopen(cache, "a")) {
      std::fprintf(f, "{\"key\": \"%s\", \"stage_kb\": %d, \"group_ctas\": %d}\n", key.c_str(),
                   h->prm.stage_kb, h->prm.group_ctas);
      std::fclose(f);
    }
  }
  if (stage_kb) *stage_kb = h->stage_bytes / 1024;
  if (group_ctas) *group_ctas = h->small ? -h->small : h->G;
  if (out != BT_OK) return out;
  // leave x with a solve in the chosen shape
  if ((out = solve()) != BT_OK) return out;
  return cudaStreamSynchronize(st) == cudaSuccess ? BT_OK : BT_ERR_CUDA;
}

bt_status bt_set_history(bt_handle h, double* hist, int len) {
  if (!h || len < 0 || (len > 0 && !hist)) return BT_ERR_ARG;
  h->hist = len > 0 ? hist : nullptr;
  h->hist_len = len;
  return BT_OK;
}

// Smallest eigenvalue of the symmetric tridiagonal (d, e) by bisection on its
// Sturm count (the number of eigenvalues below x is the number of negative
// pivots of T - x I).
static double tridiag_min_eig(const std::vector<double>& d, const std::vector<double>& e) {
  const int K = (int)d.size();
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < K; ++i) {  // Gershgorin bounds
    const double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < K ? std::fabs(e[i]) : 0.0);
    lo = std::min(lo, d[i] - r);
    hi = std::max(hi, d[i] + r);
  }
  const auto below = [&](double x) {
    int cnt = 0;
    double q = 1.0;
    for (int i = 0; i < K; ++i) {
      q = d[i] - x - (i > 0 ? e[i - 1] * e[i - 1] / q : 0.0);
      if (q == 0.0) q = -1e-300;
      if (q < 0.0) ++cnt;
    }
    return cnt;
  };
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, std::fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (below(mid) >= 1) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

bt_status bt_ritz_rho(bt_handle h, const double* b, int iters, double* rho) {
  Range nvtx_range("bt_ritz_rho");
  if (!h || !b || !rho || iters < 2) return BT_ERR_ARG;
  if (h->variant == 1 || h->prm.a != 1.0) return BT_ERR_PARAM;  // M^-1 S = I - H_opt at m = 1 needs a = 1
  cudaStream_t st = h->stream;
  const size_t len = (size_t)std::max<long long>(h->total_vec, 1);
  const size_t hl = (size_t)h->B * iters * 3;
  char* buf = nullptr;
  if (cudaMallocAsync((void**)&buf, (len + hl) * sizeof(double), st) != cudaSuccess) return BT_ERR_ALLOC;
  double* x = reinterpret_cast<double*>(buf);
  double* hist = x + len;
  std::vector<double> hh(hl, 0.0);
  bt_status out = BT_OK;
  if (cudaMemsetAsync(hist, 0, hl * sizeof(double), st) != cudaSuccess) out = BT_ERR_CUDA;
  if (out == BT_OK) {
    // `iters` iterations of PCG with M^-1 = G_opt (m = 1) from x = 0: one inner
    // solve for mixed handles, run to its iteration cap
    bt::KParams P = base_kparams(h);
    P.op = bt::kOpSolve;
    P.m = 1;
    P.bvec = b;
    P.xvec = x;
    P.tol = 0.0;
    P.tol_inner = 1e-300;
    P.maxit = iters;
    P.max_outer = 1;
    P.use_x0 = 0;
    P.hist = hist;
    P.hist_len = iters;
    out = launch(h, P);
  }
  if (out == BT_OK && (cudaMemcpyAsync(hh.data(), hist, hl * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                       cudaStreamSynchronize(st) != cudaSuccess))
    out = BT_ERR_CUDA;
  cudaFreeAsync(buf, st);
  if (out != BT_OK) return out;
  for (int k = 0; k < h->B; ++k) {
    // Lanczos tridiagonal of the preconditioned operator from the CG scalars:
    // T_00 = 1/alpha_0, T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1},
    // T_j,j-1 = sqrt(beta_{j-1})/alpha_{j-1}
    std::vector<double> d, e;
    const double* hk = hh.data() + (size_t)k * iters * 3;
    for (int j = 0; j < iters; ++j) {
      const double a = hk[3 * j + 1];
      if (!(a > 0.0) || !std::isfinite(a)) break;
      if (j == 0) {
        d.push_back(1.0 / a);
      } else {
        const double ap = hk[3 * (j - 1) + 1], bp = hk[3 * (j - 1) + 2];
        if (!(bp >= 0.0)) break;
        d.push_back(1.0 / a + bp / ap);
        e.push_back(std::sqrt(bp) / ap);
      }
    }
    rho[k] = d.empty() ? 0.0 : 1.0 - tridiag_min_eig(d, e);
  }
  return BT_OK;
}

bt_status bt_estimate_rho(bt_handle h, int iters, double* rho) {
  Range nvtx_range("bt_estimate_rho");
  if (!h || !rho || iters < 1) return BT_ERR_ARG;
  if (h->variant == 1 || h->prm.a != 1.0) return BT_ERR_PARAM;  // H_opt = I - G_opt S holds at a = 1
  cudaStream_t st = h->stream;
  const size_t len = (size_t)std::max<long long>(h->total_vec, 1);
  char* buf = nullptr;
  const size_t bytes = (3 * len + (size_t)h->B) * sizeof(double);
  if (cudaMallocAsync((void**)&buf, bytes, st) != cudaSuccess) return BT_ERR_ALLOC;
  double* v = reinterpret_cast<double*>(buf);
  double* w = v + len;
  double* u = w + len;
  double* est = u + len;
  bt_status out = BT_OK;
  bt::k_rho_step<<<h->B, 256, 0, st>>>(h->d_inst, v, u, est, 1);
  if (cudaGetLastError() != cudaSuccess) out = BT_ERR_CUDA;
  for (int k = 0; k < iters && out == BT_OK; ++k) {
    if ((out = run_op(h, bt::kOpSpmv64, v, w)) != BT_OK) break;     // w = S v (float64 blocks)
    bt::KParams P = base_kparams(h);                                 // u = G w (m = 1)
    P.op = bt::kOpApply;
    P.m = 1;
    P.bvec = w;
    P.xvec = u;
    P.tol = 0;
    P.maxit = 0;
    if ((out = launch(h, P)) != BT_OK) break;
    bt::k_rho_step<<<h->B, 256, 0, st>>>(h->d_inst, v, u, est, 0);  // v <- H v / ||H v||
    if (cudaGetLastError() != cudaSuccess) out = BT_ERR_CUDA;
  }
  if (out == BT_OK &&
      (cudaMemcpyAsync(rho, est, (size_t)h->B * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    out = BT_ERR_CUDA;
  cudaFreeAsync(buf, st);
  return out;
}

bt_status bt_params_check(const bt_params* params) {
  double alpha[BT_MAX_M];
  return check_params(params, alpha);
}

bt_status bt_alpha_chebyshev(int m, double rho, double* alpha) {
  if (!alpha || m < 1 || m > BT_MAX_M || !(rho > 0.0 && rho < 1.0)) return BT_ERR_ARG;
  return bt::alpha_chebyshev(m, rho, alpha) ? BT_OK : BT_ERR_ARG;
}

void bt_params_init(bt_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->a = 1.0;
  p->m = 2;
  p->alpha = nullptr;
  p->precision = BT_FP64;
}

const char* bt_status_string(bt_status s) {
  switch (s) {
    case BT_OK: return "ok";
    case BT_ERR_ARG: return "invalid argument";
    case BT_ERR_PARAM: return "parameter outside the admissible set";
    case BT_ERR_NOT_SPD: return "diagonal block not positive definite";
    case BT_ERR_NO_CONVERGENCE: return "no convergence within the iteration limit";
    case BT_ERR_BREAKDOWN: return "CG breakdown (p.q <= 0)";
    case BT_ERR_NONFINITE: return "non-finite value";
    case BT_ERR_TIMEOUT: return "device loop exceeded its cycle budget";
    case BT_ERR_CUDA: return "CUDA runtime error";
    case BT_ERR_ALLOC: return "device allocation failed";
    case BT_ERR_STATE: return "call not valid for this handle";
  }
  return "unknown status";
}

bt_status bt_setup(int N, int n, const double* D, const double* O, const bt_params* params, bt_handle* out) {
  Range nvtx_range("bt_setup");
  if (!out) return BT_ERR_ARG;
  *out = nullptr;
  if (N < 1 || n < 1 || n > BT_MAX_BLOCK || !D || (N > 1 && !O)) return BT_ERR_ARG;
  double alpha[BT_MAX_M];
  bt_status s = check_params(params, alpha);
  if (s != BT_OK) return s;
  bt_ctx* h = new_ctx(params);
  std::memcpy(h->alpha, alpha, sizeof(alpha));
  h->batched = false;
  h->B = 1;
  h->N = {N};
  h->n = {n};
  h->d_off = {0};
  h->o_off = {0};
  s = setup_common(h, D, O);
  if (s != BT_OK && s != BT_ERR_NOT_SPD) {
    free_all(h);
    delete h;
    return s;
  }
  *out = h;
  return s;
}

bt_status bt_setup_batched(int B, const int* N, const int* n, const long long* d_off, const long long* o_off,
                           const double* D, const double* O, const bt_params* params, bt_handle* out) {
  Range nvtx_range("bt_setup_batched");
  if (!out) return BT_ERR_ARG;
  *out = nullptr;
  if (B < 1 || !N || !n || !d_off || !o_off || !D) return BT_ERR_ARG;
  bool needO = false;
  for (int k = 0; k < B; ++k) {
    if (N[k] < 1 || n[k] < 1 || n[k] > BT_MAX_BLOCK || d_off[k] < 0 || o_off[k] < 0) return BT_ERR_ARG;
    if (N[k] > 1) needO = true;
  }
  if (needO && !O) return BT_ERR_ARG;
  double alpha[BT_MAX_M];
  bt_status s = check_params(params, alpha);
  if (s != BT_OK) return s;
  bt_ctx* h = new_ctx(params);
  std::memcpy(h->alpha, alpha, sizeof(alpha));
  h->batched = true;
  h->B = B;
  h->N.assign(N, N + B);
  h->n.assign(n, n + B);
  h->d_off.assign(d_off, d_off + B);
  h->o_off.assign(o_off, o_off + B);
  s = setup_common(h, D, O);
  if (s != BT_OK && s != BT_ERR_NOT_SPD) {
    free_all(h);
    delete h;
    return s;
  }
  *out = h;
  return s;
}

bt_status bt_refactor(bt_handle h, const double* D, const double* O) {
  Range nvtx_range("bt_refactor");
  if (!h || !D || (h->maxN > 1 && !O)) return BT_ERR_ARG;
  return launch_setup_kernels(h, D, O);
}

bt_status bt_lqr_refactor(bt_handle h, const int* m, const double* A, const double* Bm, const double* Q,
                          const double* R, const double* q, const double* r, const double* c, double* gamma,
                          int* bad_inst, int* bad_row) {
  Range nvtx_range("bt_lqr_refactor");
  if (!h || !m || !gamma) return BT_ERR_ARG;
  if (!h->mixed || h->variant != 0 || h->prm.mixed_strict_fp64) return BT_ERR_STATE;
  if (h->maxn > 48) return BT_ERR_ARG;
  cudaStream_t st = h->stream;
  if (cudaMemsetAsync(h->d_fail_key, 0xff, sizeof(unsigned long long), st)) return BT_ERR_CUDA;
  // the formation's scratch (W = L^-1 of every Q_k and R_k) is kept by the
  // handle: no allocation per call, and bt_lqr_recover_factored reads it
  const size_t need = bt_lqr_handle_bytes(h->B, h->N.data(), h->n.data(), m);
  if (need == 0) return BT_ERR_ARG;
  h->lqr_valid = false;
  if (need > h->lqr_bytes) {
    if (h->lqr_buf) {
      cudaStreamSynchronize(st);
      cudaFree(h->lqr_buf);
      h->bytes -= h->lqr_bytes;
    }
    h->lqr_buf = nullptr;
    h->lqr_bytes = 0;
    if (cudaMalloc(&h->lqr_buf, need) != cudaSuccess) {
      h->lqr_buf = nullptr;
      cudaGetLastError();
      return BT_ERR_ALLOC;
    }
    h->lqr_bytes = need;
    h->bytes += need;
  }
  const bt_status s = bt_lqr_schur_handle(h->B, h->N.data(), h->n.data(), m, A, Bm, Q, R, q, r, c, gamma, h->d_inst,
                                          h->D64, h->O64, h->D32, h->O32, h->Dinv32, st, bad_inst, bad_row,
                                          h->lqr_buf, h->lqr_bytes, nullptr);
  if (s != BT_OK) return s;
  // D_k^-1 from the float32 copy the formation left in the handle (float64
  // refactor of refused rows, as in bt_refactor), then E and the H blocks
  bt::SetupParams sp{};
  sp.inst = h->d_inst;
  sp.rows = h->d_rows;
  sp.nrows = h->total_rows;
  sp.D64 = h->D64; sp.O64 = h->O64; sp.Dinv64 = h->Dinv64; sp.E64 = h->E64;
  sp.Hd64 = h->Hd64; sp.Hu64 = h->Hu64; sp.Hl64 = h->Hl64;
  sp.D32 = h->D32; sp.O32 = h->O32; sp.Dinv32 = h->Dinv32; sp.E32 = h->E32;
  sp.Hd32 = h->Hd32; sp.Hu32 = h->Hu32; sp.Hl32 = h->Hl32;
  sp.fam_a = 1.0;
  sp.want32 = 1;
  sp.want64 = 1;
  sp.fail_key = h->d_fail_key;
  sp.fail_piv = h->d_fail_piv;
  sp.retry = h->d_retry;
  sp.segs = h->d_segs;
  sp.nsegs = h->nsegs;
  set_classes(h, sp);
  sp.copied = 1;
  if (bt_status e = cuda_st(bt_launch_setup(&sp, 1, h->prm.m, h->maxn, st)); e != BT_OK) return e;
  const bt_status e = read_setup_status(h);
  if (e == BT_OK) {
    h->lqr_valid = true;
    h->lqr_m.assign(m, m + h->B);
  }
  return e;
}

bt_status bt_lqr_recover_factored(bt_handle h, const int* m, const double* A, const double* Bm, const double* q,
                                  const double* r, const double* lambda, double* x, double* u) {
  Range nvtx_range("bt_lqr_recover_factored");
  if (!h || !m) return BT_ERR_ARG;
  if (!h->lqr_valid || !std::equal(h->lqr_m.begin(), h->lqr_m.end(), m)) return BT_ERR_STATE;
  return bt_lqr_recover_w_run(h->B, h->N.data(), h->n.data(), m, A, Bm, q, r, lambda, x, u, h->lqr_buf, h->stream);
}

bt_status bt_setup_status(bt_handle h) {
  if (!h) return BT_ERR_ARG;
  return read_setup_status(h);
}

bt_status bt_apply_precond(bt_handle h, const double* r, double* z) {
  Range nvtx_range("bt_apply_precond");
  if (!h || !r || !z) return BT_ERR_ARG;
  bt_status s = run_op(h, bt::kOpApply, r, z);
  if (s != BT_OK) return s;
  return cuda_st(cudaStreamSynchronize(h->stream));
}

bt_status bt_spmv(bt_handle h, const double* x, double* y) {
  if (!h || !x || !y) return BT_ERR_ARG;
  bt_status s = run_op(h, bt::kOpSpmv64, x, y);
  if (s != BT_OK) return s;
  return cuda_st(cudaStreamSynchronize(h->stream));
}

bt_status bt_spmv_f32(bt_handle h, const double* x, double* y) {
  if (!h || !x || !y) return BT_ERR_ARG;
  if (!h->mixed) return BT_ERR_STATE;
  bt_status s = run_op(h, bt::kOpSpmv32, x, y);
  if (s != BT_OK) return s;
  return cuda_st(cudaStreamSynchronize(h->stream));
}

static bt_status solve_launch(bt_handle h, const double* b, double* x, double tol, int maxit) {
  if (!(tol >= 0.0) || maxit < 0) return BT_ERR_ARG;
  if (h->small) {
    const double* blk[7] = {h->D64, h->O64, h->Dinv64, h->E64, h->Hd64, h->Hu64, h->Hl64};
    const float* blk32[7] = {h->D32, h->O32, h->Dinv32, h->E32, h->Hd32, h->Hu32, h->Hl32};
    const int n = h->n[0];
    return cuda_st(bt_small_launch(blk, h->mixed ? blk32 : nullptr, h->N[0], n, (int)rup((long long)n * n, 2),
                                   bt::slot32(n), h->prm.m, h->alpha, b, x, h->prm.use_x0, tol, h->prm.tol_inner,
                                   h->prm.max_outer > 0 ? h->prm.max_outer : 30, maxit,
                                   h->prm.cycle_budget > 0 ? h->prm.cycle_budget : (1ll << 34), h->hist,
                                   h->hist_len, h->d_iters, h->d_status, h->d_outer, h->d_resid, h->d_errval,
                                   h->prm.mixed_strict_fp64, h->small, h->stream));
  }
  bt::KParams P = base_kparams(h);
  P.op = bt::kOpSolve;
  P.bvec = b;
  P.xvec = x;
  P.tol = tol;
  P.maxit = maxit;
  return launch(h, P);
}

bt_status bt_pcg_solve(bt_handle h, const double* b, double* x, double tol, int maxit, int* iters) {
  Range nvtx_range("bt_pcg_solve");
  if (!h || !b || !x) return BT_ERR_ARG;
  if (h->batched) return BT_ERR_STATE;
  bt_status s = solve_launch(h, b, x, tol, maxit);
  if (s != BT_OK) return s;
  int it = 0;
  s = collect(h, &it, nullptr, true);
  if (iters) *iters = it;
  return s;
}

bt_status bt_pcg_solve_async(bt_handle h, const double* b, double* x, double tol, int maxit, int* d_iters,
                             int* d_status) {
  Range nvtx_range("bt_pcg_solve_async");
  if (!h || !b || !x) return BT_ERR_ARG;
  if (h->batched) return BT_ERR_STATE;
  bt_status s = solve_launch(h, b, x, tol, maxit);
  if (s != BT_OK) return s;
  if (d_iters && cudaMemcpyAsync(d_iters, h->d_iters, sizeof(int), cudaMemcpyDeviceToDevice, h->stream))
    return BT_ERR_CUDA;
  if (d_status && cudaMemcpyAsync(d_status, h->d_status, sizeof(int), cudaMemcpyDeviceToDevice, h->stream))
    return BT_ERR_CUDA;
  return BT_OK;
}

bt_status bt_pcg_solve_batched(bt_handle h, const double* b, double* x, const long long* vec_off, double tol,
                               int maxit, int* iters, int* status) {
  Range nvtx_range("bt_pcg_solve_batched");
  if (!h || !b || !x) return BT_ERR_ARG;
  if (!h->batched) return BT_ERR_STATE;
  if (vec_off) {
    bool same = true;
    for (int k = 0; k < h->B; ++k) same &= (vec_off[k] == h->vec_off[k]);
    if (!same) {
      // re-pack the descriptors with the new vector offsets
      std::vector<bt::InstDesc> inst(h->B);
      cudaMemcpy(inst.data(), h->d_inst, h->B * sizeof(bt::InstDesc), cudaMemcpyDeviceToHost);
      for (int k = 0; k < h->B; ++k) {
        if (vec_off[k] < 0) return BT_ERR_ARG;
        inst[k].vec = vec_off[k];
        h->vec_off[k] = vec_off[k];
      }
      if (cudaMemcpy(h->d_inst, inst.data(), h->B * sizeof(bt::InstDesc), cudaMemcpyHostToDevice))
        return BT_ERR_CUDA;
    }
  }
  bt_status s = solve_launch(h, b, x, tol, maxit);
  if (s != BT_OK) return s;
  return collect(h, iters, status, true);
}

bt_status bt_pcg_solve_batched_async(bt_handle h, const double* b, double* x, double tol, int maxit,
                                     int* d_iters, int* d_status) {
  Range nvtx_range("bt_pcg_solve_batched_async");
  if (!h || !b || !x) return BT_ERR_ARG;
  if (!h->batched) return BT_ERR_STATE;
  bt_status s = solve_launch(h, b, x, tol, maxit);
  if (s != BT_OK) return s;
  if (d_iters &&
      cudaMemcpyAsync(d_iters, h->d_iters, h->B * sizeof(int), cudaMemcpyDeviceToDevice, h->stream))
    return BT_ERR_CUDA;
  if (d_status &&
      cudaMemcpyAsync(d_status, h->d_status, h->B * sizeof(int), cudaMemcpyDeviceToDevice, h->stream))
    return BT_ERR_CUDA;
  return BT_OK;
}

bt_status bt_graph_capture_batched(bt_handle h, const double* b, double* x, double tol, int maxit, int* d_iters,
                                   int* d_status) {
  Range nvtx_range("bt_graph_capture_batched");
  if (!h) return BT_ERR_ARG;
  if (!h->batched) return BT_ERR_STATE;
  if (!h->stream) return BT_ERR_ARG;  // the legacy default stream cannot be captured
  if (h->graph) cudaGraphExecDestroy(h->graph);
  if (h->graph_src) cudaGraphDestroy(h->graph_src);
  h->graph = nullptr;
  h->graph_src = nullptr;
  // make sure the kernel attributes are set before capture
  int occ = 0;
  bt_persistent_occupancy(h->mixed, h->variant, h->smem, &occ);
  if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal)) return BT_ERR_CUDA;
  bt_status s = bt_pcg_solve_batched_async(h, b, x, tol, maxit, d_iters, d_status);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  if (s != BT_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e) return BT_ERR_CUDA;
  h->graph_src = g;
  if (cudaGraphInstantiate(&h->graph, g, 0)) return BT_ERR_CUDA;
  return BT_OK;
}

bt_status bt_graph_capture_refactor_solve(bt_handle h, const double* D, const double* O, const double* b, double* x,
                                          double tol, int maxit, int* d_iters, int* d_status) {
  Range nvtx_range("bt_graph_capture_refactor_solve");
  if (!h || !D || (h->maxN > 1 && !O)) return BT_ERR_ARG;
  if (!h->batched) return BT_ERR_STATE;
  if (!h->stream) return BT_ERR_ARG;  // the legacy default stream cannot be captured
  if (h->graph) cudaGraphExecDestroy(h->graph);
  if (h->graph_src) cudaGraphDestroy(h->graph_src);
  h->graph = nullptr;
  h->graph_src = nullptr;
  // kernel attributes were set when bt_setup_batched launched the same kernels
  int occ = 0;
  bt_persistent_occupancy(h->mixed, h->variant, h->smem, &occ);
  if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal)) return BT_ERR_CUDA;
  bt_status s = launch_setup_kernels(h, D, O);
  if (s == BT_OK) s = bt_pcg_solve_batched_async(h, b, x, tol, maxit, d_iters, d_status);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  if (s != BT_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e) return BT_ERR_CUDA;
  h->graph_src = g;
  if (cudaGraphInstantiate(&h->graph, g, 0)) return BT_ERR_CUDA;
  return BT_OK;
}

bt_status bt_graph_launch(bt_handle h) {
  if (!h || !h->graph) return BT_ERR_STATE;
  return cuda_st(cudaGraphLaunch(h->graph, h->stream));
}

bt_status bt_solve_info(bt_handle h, int k, int* outer, double* rel_residual) {
  if (!h || k < 0 || k >= h->B) return BT_ERR_ARG;
  if ((int)h->h_outer.size() != h->B) return BT_ERR_STATE;
  if (outer) *outer = h->h_outer[k];
  if (rel_residual) *rel_residual = h->h_resid[k];
  return BT_OK;
}

bt_status bt_adjoint_blocks(bt_handle h, const double* x, const double* g, double* gD, double* gO) {
  Range nvtx_range("bt_adjoint_blocks");
  if (!h || !x || !g || !gD) return BT_ERR_ARG;
  if (!gO && h->maxN > 1) return BT_ERR_ARG;
  bt::AdjParams a{};
  a.inst = h->d_inst;
  a.rows = h->d_rows;
  a.nrows = h->total_rows;
  a.d_off = h->d_doff;
  a.o_off = h->d_ooff;
  a.x = x;
  a.g = g;
  a.gD = gD;
  a.gO = gO;
  return cuda_st(bt_launch_adjoint(&a, h->stream));
}

bt_status bt_pcg_solve_multi(bt_handle h, const double* B, double* X, int nrhs, double tol, int maxit, int* iters,
                             int* status) {
  Range nvtx_range("bt_pcg_solve_multi");
  if (!h || !B || !X) return BT_ERR_ARG;
  if (h->batched) return BT_ERR_STATE;
  if (!h->mixed) return BT_ERR_STATE;
  if (h->variant != 0) return BT_ERR_PARAM;  // the many-RHS engine: the optimum with stored H only
  if (nrhs < 1 || nrhs > 64 || !(tol >= 0.0) || maxit < 0) return BT_ERR_ARG;
  const int N = h->N[0], n = h->n[0];
  if (n % 4 != 0 || n > 64) return BT_ERR_ARG;  // 16 row groups of 4 at most (BT_MAX_BLOCK)
  const int kJ = 64;
  if (!h->mr_vec[16]) {  // the last entry: a partly allocated workspace is allocated again
    const size_t cnt = (size_t)N * n * kJ;
    bt_status s;
    double* d = nullptr;
    float* f = nullptr;
    for (int i = 0; i < 3; ++i) {  // B64, X64, R64
      if ((s = dalloc(h, &d, cnt)) != BT_OK) return s;
      h->mr_vec[i] = d;
    }
    for (int i = 3; i < 11; ++i) {  // Xin, R, P, Q, Y0, Ya, Yb, Z
      if ((s = dalloc(h, &f, cnt)) != BT_OK) return s;
      h->mr_vec[i] = f;
    }
    // one CTA per SM in either engine (both need more than half the shared memory)
    h->mr_G = std::max(1, std::min(h->sms, N));
    double* red = nullptr;
    if ((s = dalloc(h, &red, (size_t)2 * h->mr_G * kJ)) != BT_OK) return s;
    h->mr_vec[11] = red;
    int* ctl = nullptr;
    if ((s = dalloc(h, &ctl, 64)) != BT_OK) return s;
    h->mr_vec[12] = ctl;
    int* res_i = nullptr;
    if ((s = dalloc(h, &res_i, 3 * kJ)) != BT_OK) return s;
    h->mr_vec[13] = res_i;
    double* res_d = nullptr;
    if ((s = dalloc(h, &res_d, kJ)) != BT_OK) return s;
    h->mr_vec[14] = res_d;
    if ((s = dalloc(h, &f, cnt)) != BT_OK) return s;  // second p buffer
    h->mr_vec[15] = f;
    if ((s = dalloc(h, &f, cnt)) != BT_OK) return s;  // second r buffer
    h->mr_vec[16] = f;
  }
  // engine: tensor cores (3xTF32) where supported, unless the caller asks for SIMT
  const int tc_ok = bt_mrhs_tc_supported(n);
  if (h->prm.mrhs_engine == 2 && !tc_ok) return BT_ERR_ARG;
  const int tc = (h->prm.mrhs_engine == 2 || (h->prm.mrhs_engine == 0 && tc_ok)) ? 1 : 0;
  const float* blk32[7] = {h->D32, h->O32, h->Dinv32, h->E32, h->Hd32, h->Hu32, h->Hl32};
  const int bs32 = bt::slot32(n), bs64 = (int)rup((long long)n * n, 2);
  if (tc) {
    if (!h->mr_img[8]) {
      for (int i = 0; i < 9; ++i) {
        bt_status s2 = dalloc(h, &h->mr_img[i], (size_t)N * n * n * 2);  // [hi | lo] TF32 parts
        if (s2 != BT_OK) return s2;
      }
    }
    // the images follow the handle's current blocks (a refactor may have changed them)
    if (bt_mrhs_images(N, n, h->prm.m, blk32, bs32, h->mr_img, h->stream) != cudaSuccess) return BT_ERR_CUDA;
  }
  h->mr_smem = bt_mrhs_smem_bytes(n, tc);
  {
    int occ = 0;
    if (bt_mrhs_occupancy(h->mr_smem, tc, &occ) != cudaSuccess || occ < 1) return BT_ERR_CUDA;
    if (h->mr_G > h->sms * occ) return BT_ERR_CUDA;
  }
  if (cudaMemsetAsync(h->mr_vec[12], 0, 64 * sizeof(int), h->stream)) return BT_ERR_CUDA;
  const double tin = h->prm.tol_inner > 0 ? h->prm.tol_inner : 1e-5;  // measured best for the 64-column solve
  const int mo = h->prm.max_outer > 0 ? h->prm.max_outer : 30;
  const long long budget = h->prm.cycle_budget > 0 ? h->prm.cycle_budget : (1ll << 36);
  cudaError_t e = bt_mrhs_solve_launch(N, n, h->prm.m, h->alpha, blk32, h->D64, h->O64, bs32, bs64, h->mr_vec,
                                       tc ? h->mr_img : nullptr, tol, tin, maxit, mo, budget, h->mr_G, nrhs, B, X,
                                       h->mr_smem, h->stream);
  if (e != cudaSuccess) return BT_ERR_CUDA;
  std::vector<int> ri(3 * kJ);
  std::vector<double> rd(kJ);
  if (cudaMemcpyAsync(ri.data(), h->mr_vec[13], 3 * kJ * sizeof(int), cudaMemcpyDeviceToHost, h->stream) ||
      cudaMemcpyAsync(rd.data(), h->mr_vec[14], kJ * sizeof(double), cudaMemcpyDeviceToHost, h->stream) ||
      cudaStreamSynchronize(h->stream))
    return BT_ERR_CUDA;
  bt_status first = BT_OK;
  for (int j = 0; j < nrhs; ++j) {
    if (iters) iters[j] = ri[j];
    if (status) status[j] = ri[kJ + j];
    if (ri[kJ + j] != BT_OK && first == BT_OK) first = static_cast<bt_status>(ri[kJ + j]);
  }
  h->mr_resid.assign(rd.begin(), rd.begin() + nrhs);
  h->mr_outer = ri[2 * kJ];
  return first;
}

bt_status bt_multi_info(bt_handle h, int j, int* outer, double* rel_residual) {
  if (!h || j < 0 || j >= (int)h->mr_resid.size()) return BT_ERR_ARG;
  if (outer) *outer = h->mr_outer;
  if (rel_residual) *rel_residual = h->mr_resid[j];
  return BT_OK;
}

bt_status bt_last_error(bt_handle h, int* instance, int* block, double* value) {
  if (!h) return BT_ERR_ARG;
  if (instance) *instance = h->err_inst;
  if (block) *block = h->err_blk;
  if (value) *value = h->err_val;
  return BT_OK;
}

long long bt_device_bytes(bt_handle h) { return h ? (long long)h->bytes : 0; }

void bt_destroy(bt_handle h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  free_all(h);
  delete h;
}

}  // extern "C"
