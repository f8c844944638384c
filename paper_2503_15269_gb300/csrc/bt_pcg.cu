// Persistent PCG kernels of the optimum (a = 1, stored H_opt) and the host
// launchers of every persistent kernel.  The kernel template lives in
// bt_pcg_kernel.cuh; the kernels of a general member of the family (a < 1)
// and of the matrix-free H_opt are instantiated in bt_pcg_gen.cu and
// bt_pcg_mf.cu, separate translation units compiled in parallel.
#include "bt_pcg_kernel.cuh"

namespace bt {
template __global__ void bt_persistent_kernel<float, 0>(const __grid_constant__ KParams P);
template __global__ void bt_persistent_kernel<double, 0>(const __grid_constant__ KParams P);
}  // namespace bt

extern "C" const void* bt_persistent_fn_gen(int mt_is_float);
extern "C" int bt_persistent_smem_fixed_gen();
extern "C" const void* bt_persistent_fn_mf(int mt_is_float);

// variant: 0 = optimum with stored H_opt, 1 = general member, 2 = matrix-free H_opt
static const void* persistent_fn(int mt_is_float, int variant) {
  if (variant == 1) return bt_persistent_fn_gen(mt_is_float);
  if (variant == 2) return bt_persistent_fn_mf(mt_is_float);
  return mt_is_float ? (const void*)bt::bt_persistent_kernel<float, 0>
                     : (const void*)bt::bt_persistent_kernel<double, 0>;
}

// Host-side entry used by bt_api.cu and bt_noalloc.cu; P->variant selects the
// kernels.
extern "C" cudaError_t bt_launch_persistent(const bt::KParams* P, int grid, int smem_bytes, int mt_is_float,
                                            int cooperative, cudaStream_t stream) {
  const void* fn = persistent_fn(mt_is_float, P->variant);
  cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (err != cudaSuccess) return err;
  void* args[] = {(void*)P};
  if (cooperative) return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(bt::kThreads), args, smem_bytes, stream);
  return cudaLaunchKernel(fn, dim3(grid), dim3(bt::kThreads), args, smem_bytes, stream);
}

extern "C" int bt_persistent_smem_fixed(int variant) {
  return variant == 1 ? bt_persistent_smem_fixed_gen() : bt::smem_fixed_bytes<false>();
}

extern "C" cudaError_t bt_persistent_occupancy(int mt_is_float, int variant, int smem_bytes, int* blocks_per_sm) {
  const void* fn = persistent_fn(mt_is_float, variant);
  cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (err != cudaSuccess) return err;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, bt::kThreads, smem_bytes);
}
