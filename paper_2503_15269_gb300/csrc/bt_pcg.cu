// Persistent PCG kernels of the optimum (a = 1) and the host launchers of
// every persistent kernel.  The kernel template lives in bt_pcg_kernel.cuh;
// the kernels of a general member of the family (a < 1) are instantiated in
// bt_pcg_gen.cu, a separate translation unit compiled in parallel.
#include "bt_pcg_kernel.cuh"

namespace bt {
template __global__ void bt_persistent_kernel<float, false>(const __grid_constant__ KParams P);
template __global__ void bt_persistent_kernel<double, false>(const __grid_constant__ KParams P);
}  // namespace bt

extern "C" const void* bt_persistent_fn_gen(int mt_is_float);
extern "C" int bt_persistent_smem_fixed_gen();

static const void* persistent_fn(int mt_is_float, int general) {
  if (general) return bt_persistent_fn_gen(mt_is_float);
  return mt_is_float ? (const void*)bt::bt_persistent_kernel<float, false>
                     : (const void*)bt::bt_persistent_kernel<double, false>;
}

// Host-side entry used by bt_api.cu and bt_noalloc.cu; P->general selects the
// kernels of the general member.
extern "C" cudaError_t bt_launch_persistent(const bt::KParams* P, int grid, int smem_bytes, int mt_is_float,
                                            int cooperative, cudaStream_t stream) {
  const void* fn = persistent_fn(mt_is_float, P->general);
  cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (err != cudaSuccess) return err;
  void* args[] = {(void*)P};
  if (cooperative) return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(bt::kThreads), args, smem_bytes, stream);
  return cudaLaunchKernel(fn, dim3(grid), dim3(bt::kThreads), args, smem_bytes, stream);
}

extern "C" int bt_persistent_smem_fixed(int general) {
  return general ? bt_persistent_smem_fixed_gen() : bt::smem_fixed_bytes<false>();
}

extern "C" cudaError_t bt_persistent_occupancy(int mt_is_float, int general, int smem_bytes, int* blocks_per_sm) {
  const void* fn = persistent_fn(mt_is_float, general);
  cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (err != cudaSuccess) return err;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, bt::kThreads, smem_bytes);
}
