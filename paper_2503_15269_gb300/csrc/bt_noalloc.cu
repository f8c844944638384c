// bt_pcg_solve_noalloc: a single-instance solve that allocates no device
// memory.
//
// Who needs it: callers that cannot call cudaMalloc -- for example a
// real-time control loop whose memory is fixed at start-up (cudaMalloc can
// synchronise the device and takes unbounded time), or a plug-in that runs
// inside a host application which owns the GPU memory budget.  Such a caller
// passes only its inputs (D, O, b) and output (x); everything the solve needs
// besides them -- the library-layout copies of the blocks, D_i^-1, E_i, the H
// blocks, the PCG work vectors, the reduction/barrier words and the result
// words -- is carved out of one file-scope device array of fixed size,
// BT_NOALLOC_SCRATCH_BYTES, that every GPU loading the library holds until
// the process exits.
//
// It runs the same kernels as bt_setup + bt_pcg_solve (setup kernels, then
// the persistent PCG kernel) on that scratch.  Every call shares the array
// and leaves its contents behind; what must start at zero (control words,
// padding slots of the block arrays) is cleared at the start of each call.
// Calls that overlap on the GPU (two streams, or two host threads) race on
// the array: issue them one after another.
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "../../include/bt.h"
#include "bt_alpha.h"
#include "bt_common.cuh"

extern "C" cudaError_t bt_launch_persistent(const bt::KParams* P, int grid, int smem_bytes, int mt_is_float,
                                            int cooperative, cudaStream_t stream);
extern "C" int bt_persistent_smem_fixed(int variant);
extern "C" cudaError_t bt_persistent_occupancy(int mt_is_float, int variant, int smem_bytes, int* blocks_per_sm);
extern "C" cudaError_t bt_launch_setup(const bt::SetupParams* P, int mixed, int m, int maxn, cudaStream_t st);

static __device__ __align__(256) unsigned char g_bt_noalloc_scratch[BT_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};
unsigned long long g_ctx_id[kMaxDevices] = {};

// Device address of the scratch array for the current device, looked up
// (cudaGetSymbolAddress, with that device current) on the first call in each
// CUDA context of the device and cached under the context's unique id: a
// cudaDeviceReset or a new primary context loads the module afresh, and the
// next call then looks the address up again instead of using a stale one.
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  e = cudaSetDevice(dev);  // initialises the device's primary context and makes it current
  if (e != cudaSuccess) return e;
  // the driver API through the runtime's entry-point lookup (no link-time
  // dependency on the driver library)
  using CtxGetCurrent = CUresult (*)(CUcontext*);
  using CtxGetId = CUresult (*)(CUcontext, unsigned long long*);
  static CtxGetCurrent get_current = nullptr;
  static CtxGetId get_id = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!get_current || !get_id) {
      void* f1 = nullptr;
      void* f2 = nullptr;
      cudaDriverEntryPointQueryResult q1{}, q2{};
      if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
          cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
          q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
        return cudaErrorSymbolNotFound;
      get_current = reinterpret_cast<CtxGetCurrent>(f1);
      get_id = reinterpret_cast<CtxGetId>(f2);
    }
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return cudaErrorDeviceUninitialized;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev] || g_ctx_id[dev] != id) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_bt_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<unsigned char*>(p);
    g_ctx_id[dev] = id;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

// Fill the instance descriptor and the row table, clear the control words.
__global__ void k_noalloc_init(bt::InstDesc* inst, bt::RowRef* rows, long long* offs, int* order, int N, int n,
                               int bs32, int bs64, int* ctl, int nctl, unsigned long long* fail_key) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) {
    *order = 0;
    inst->N = N;
    inst->n = n;
    inst->bs32 = bs32;
    inst->bs64 = bs64;
    inst->off32 = 0;
    inst->off64 = 0;
    inst->vec = 0;
    offs[0] = 0;
    offs[1] = 0;
    *fail_key = ~0ull;
  }
  if (t < nctl) ctl[t] = 0;
  for (int i = t; i < N; i += gridDim.x * blockDim.x) rows[i] = bt::RowRef{0, i};
}

struct Carve {
  size_t off = 0;
  template <typename T>
  T* take(unsigned char* base, size_t count) {
    T* p = reinterpret_cast<T*>(base + off);
    off += (count * sizeof(T) + 255) / 256 * 256;
    return p;
  }
};

inline long long rup(long long v, long long a) { return (v + a - 1) / a * a; }

}  // namespace

extern "C" bt_status bt_pcg_solve_noalloc(int N, int n, const double* D, const double* O, const double* b,
                                          double* x, double tol, int maxit, const bt_params* p, int* iters) {
  if (N < 1 || n < 1 || n > BT_MAX_BLOCK || !D || (N > 1 && !O) || !b || !x || !p) return BT_ERR_ARG;
  if (!(tol >= 0.0) || maxit < 0) return BT_ERR_ARG;
  // parameters: bt_setup's admissible set, restricted to the optimum a = 1
  // (the static buffer has no room for the +-1 blocks of a general H_ab)
  if (p->a != 1.0 || p->h_matrix_free != 0 || p->m < 1 || p->m > BT_MAX_M) return BT_ERR_PARAM;
  if (p->precision != BT_FP64 && p->precision != BT_MIXED) return BT_ERR_PARAM;
  if (p->tol_inner < 0.0 || p->tol_inner >= 1.0 || p->max_outer < 0 || p->cycle_budget < 0) return BT_ERR_PARAM;
  if (p->mixed_strict_fp64 != 0 && p->mixed_strict_fp64 != 1) return BT_ERR_PARAM;
  double alpha[BT_MAX_M] = {0};
  for (int j = 0; j < p->m; ++j) {
    const double a = p->alpha ? p->alpha[j] : 1.0;
    if (!std::isfinite(a)) return BT_ERR_PARAM;
    alpha[j] = a;
  }
  if (alpha[0] != 1.0) return BT_ERR_PARAM;
  if (!bt::alpha_positive_on_unit_interval(alpha, p->m)) return BT_ERR_PARAM;
  const bool mixed = p->precision == BT_MIXED;
  const int m = p->m;
  cudaStream_t st = static_cast<cudaStream_t>(p->stream);

  int dev = 0, sms = 0, smem_optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return BT_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);

  // launch configuration (same rules as a handle made by bt_setup)
  const int bs32 = bt::slot32(n);
  const int bs64 = (int)rup((long long)n * n, 2);
  const long long bsb = mixed ? (long long)bs32 * 4 : (long long)bs64 * 8;
  long long sb = p->stage_kb > 0 ? (long long)p->stage_kb * 1024 : 80 * 1024;
  sb = std::max(sb, rup(std::max(5 * bsb, 3 * (long long)bs64 * 8), 128));
  const int fixed = bt_persistent_smem_fixed(0);
  int vslot = mixed ? 9 * 1024 : 18 * 1024;
  const long long per_cta = std::min<long long>(smem_optin, 228 * 1024 - 1024);
  const int vslots = 4;  // vector ring slots of the optimum's kernel variant
  int S = (int)((per_cta - fixed - vslots * vslot) / sb);
  if (S < 2) {
    vslot = 0;
    S = (int)((per_cta - fixed) / sb);
  }
  S = std::min(S, bt::kMaxStages);
  if (S < 2) return BT_ERR_ARG;
  const int smem = fixed + vslots * vslot + S * (int)sb;
  int occ = 0;
  if (bt_persistent_occupancy(mixed ? 1 : 0, 0, smem, &occ) != cudaSuccess || occ < 1) return BT_ERR_CUDA;
  int G = p->group_ctas > 0 ? p->group_ctas : (N <= 32 ? 1 : std::max(1, N / 4));
  G = std::max(1, std::min({G, sms * occ, N}));

  // carve the scratch array
  unsigned char* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return BT_ERR_CUDA;
  const long long ws_vec = rup((long long)N * n, 64);
  const bool wantH = m >= 2;
  Carve c;
  int* ctl = c.take<int>(base, 64);
  int* d_iters = c.take<int>(base, 1);
  int* d_status = c.take<int>(base, 1);
  int* d_outer = c.take<int>(base, 1);
  double* d_resid = c.take<double>(base, 1);
  double* d_errval = c.take<double>(base, 1);
  unsigned long long* fail_key = c.take<unsigned long long>(base, 1);
  bt::InstDesc* inst = c.take<bt::InstDesc>(base, 1);
  long long* offs = c.take<long long>(base, 2);
  int* order = c.take<int>(base, 1);
  bt::RowRef* rows = c.take<bt::RowRef>(base, N);
  double* fail_piv = c.take<double>(base, N);
  int* retry = mixed ? c.take<int>(base, (size_t)N + 1) : nullptr;
  double* red = c.take<double>(base, (size_t)2 * G * 4);
  const size_t blocks_begin = c.off;
  const size_t n64 = (size_t)N * bs64, n32 = (size_t)N * bs32;
  double* D64 = c.take<double>(base, n64);
  double* O64 = c.take<double>(base, n64);
  double *Dinv64 = nullptr, *E64 = nullptr, *Hd64 = nullptr, *Hu64 = nullptr, *Hl64 = nullptr;
  float *D32 = nullptr, *O32 = nullptr, *Dinv32 = nullptr, *E32 = nullptr, *Hd32 = nullptr, *Hu32 = nullptr,
        *Hl32 = nullptr;
  if (mixed) {
    D32 = c.take<float>(base, n32);
    O32 = c.take<float>(base, n32);
    Dinv32 = c.take<float>(base, n32);
    E32 = c.take<float>(base, n32);
    if (wantH) {
      Hd32 = c.take<float>(base, n32);
      Hu32 = c.take<float>(base, n32);
      Hl32 = c.take<float>(base, n32);
    }
  } else {
    Dinv64 = c.take<double>(base, n64);
    E64 = c.take<double>(base, n64);
    if (wantH) {
      Hd64 = c.take<double>(base, n64);
      Hu64 = c.take<double>(base, n64);
      Hl64 = c.take<double>(base, n64);
    }
  }
  const size_t blocks_end = c.off;
  const size_t ws_stride = (size_t)rup(10 * ws_vec * (mixed ? 4 : 8) + ws_vec * 8, 256);
  char* ws = c.take<char>(base, ws_stride);
  if (c.off > (size_t)BT_NOALLOC_SCRATCH_BYTES) return BT_ERR_ARG;  // instance too large for the scratch

  // clear what must start at zero (block arrays with their padding slots, and
  // the PCG workspace, whose padding an earlier call -- one that diverged or
  // had non-finite input -- may have left non-finite), then set up and solve
  if (cudaMemsetAsync(base + blocks_begin, 0, blocks_end - blocks_begin, st)) return BT_ERR_CUDA;
  if (cudaMemsetAsync(ws, 0, ws_stride, st)) return BT_ERR_CUDA;
  k_noalloc_init<<<std::max(1, (N + 255) / 256), 256, 0, st>>>(inst, rows, offs, order, N, n, bs32, bs64, ctl,
                                                              64, fail_key);
  if (cudaGetLastError() != cudaSuccess) return BT_ERR_CUDA;
  bt::SetupParams sp{};
  sp.fam_a = 1.0;  // the optimum: no F/K blocks, no scaling
  sp.inst = inst;
  sp.rows = rows;
  sp.nrows = N;
  sp.D = D;
  sp.O = O;
  sp.d_off = offs;
  sp.o_off = offs + 1;
  sp.D64 = D64; sp.O64 = O64; sp.Dinv64 = Dinv64; sp.E64 = E64; sp.Hd64 = Hd64; sp.Hu64 = Hu64; sp.Hl64 = Hl64;
  sp.D32 = D32; sp.O32 = O32; sp.Dinv32 = Dinv32; sp.E32 = E32; sp.Hd32 = Hd32; sp.Hu32 = Hu32; sp.Hl32 = Hl32;
  sp.want32 = mixed ? 1 : 0;
  sp.want64 = 1;
  sp.fail_key = fail_key;
  sp.fail_piv = fail_piv;
  sp.retry = p->mixed_strict_fp64 ? nullptr : retry;  // strict: every D_i factored in float64
  if (bt_launch_setup(&sp, mixed ? 1 : 0, m, n, st) != cudaSuccess) return BT_ERR_CUDA;

  bt::KParams P{};
  P.D64 = D64; P.O64 = O64; P.Dinv64 = Dinv64; P.E64 = E64; P.Hd64 = Hd64; P.Hu64 = Hu64; P.Hl64 = Hl64;
  P.D32 = D32; P.O32 = O32; P.Dinv32 = Dinv32; P.E32 = E32; P.Hd32 = Hd32; P.Hu32 = Hu32; P.Hl32 = Hl32;
  P.inst = inst;
  P.order = order;
  P.B = 1;
  P.queue = ctl;
  P.abort_flag = ctl + 1;
  P.bar = reinterpret_cast<unsigned*>(ctl + 2);
  P.red = red;
  P.bvec = b;
  P.xvec = x;
  P.op = bt::kOpSolve;
  P.mixed = mixed ? 1 : 0;
  P.scal64 = p->mixed_strict_fp64;
  P.m = m;
  for (int j = 0; j < BT_MAX_M; ++j) P.alpha[j] = alpha[j];
  P.tol = tol;
  P.tol_inner = p->tol_inner;  // 0: the kernel derives it from tol
  P.maxit = maxit;
  P.max_outer = p->max_outer > 0 ? p->max_outer : 30;
  P.use_x0 = p->use_x0;
  P.budget = p->cycle_budget > 0 ? p->cycle_budget : (1ll << 34);
  P.ws = ws;
  P.ws_stride = (long long)ws_stride;
  P.ws_vec = ws_vec;
  P.G = G;
  P.iters = d_iters;
  P.status = d_status;
  P.outer = d_outer;
  P.resid = d_resid;
  P.errval = d_errval;
  P.stages = S;
  P.stage_bytes = (int)sb;
  P.vec_slot_bytes = vslot;

  unsigned long long key = 0;
  if (cudaMemcpyAsync(&key, fail_key, sizeof(key), cudaMemcpyDeviceToHost, st)) return BT_ERR_CUDA;
  if (cudaStreamSynchronize(st)) return BT_ERR_CUDA;
  if (key != ~0ull) return BT_ERR_NOT_SPD;
  if (bt_launch_persistent(&P, G, smem, mixed ? 1 : 0, G > 1 ? 1 : 0, st) != cudaSuccess) return BT_ERR_CUDA;
  int h_it = 0, h_st = 0;
  if (cudaMemcpyAsync(&h_it, d_iters, sizeof(int), cudaMemcpyDeviceToHost, st) ||
      cudaMemcpyAsync(&h_st, d_status, sizeof(int), cudaMemcpyDeviceToHost, st) || cudaStreamSynchronize(st))
    return BT_ERR_CUDA;
  if (iters) *iters = h_it;
  return static_cast<bt_status>(h_st);
}
