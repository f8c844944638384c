// Persistent PCG kernels of a general member (a < 1, b = 1 - 2a) of the
// multi-splitting family: the kernel template of bt_pcg_kernel.cuh with H
// sweeps of kind kKB2G (five block arrays of H_ab) and the shared-memory
// region those sweeps use.  Launched through bt_launch_persistent (bt_pcg.cu).
#include "bt_pcg_kernel.cuh"

namespace bt {
template __global__ void bt_persistent_kernel<float, 1>(const __grid_constant__ KParams P);
template __global__ void bt_persistent_kernel<double, 1>(const __grid_constant__ KParams P);
}  // namespace bt

extern "C" const void* bt_persistent_fn_gen(int mt_is_float) {
  return mt_is_float ? (const void*)bt::bt_persistent_kernel<float, 1>
                     : (const void*)bt::bt_persistent_kernel<double, 1>;
}

extern "C" int bt_persistent_smem_fixed_gen() { return bt::smem_fixed_bytes<true>(); }
