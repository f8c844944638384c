// Persistent PCG kernels of the optimum (a = 1) with the matrix-free H_opt:
// H_opt = H_J^2 applied as two sweeps of kind kKJ over D^-1 and O (H_J v =
// -D^-1 (O_{i-1}^T v_{i-1} + O_i v_{i+1})), so no Hd, Hu, Hl blocks are stored
// -- for problems bound by memory capacity rather than bandwidth.  The kernel
// template of bt_pcg_kernel.cuh; launched through bt_launch_persistent.
#include "bt_pcg_kernel.cuh"

namespace bt {
template __global__ void bt_persistent_kernel<float, 2>(const __grid_constant__ KParams P);
template __global__ void bt_persistent_kernel<double, 2>(const __grid_constant__ KParams P);
}  // namespace bt

extern "C" const void* bt_persistent_fn_mf(int mt_is_float) {
  return mt_is_float ? (const void*)bt::bt_persistent_kernel<float, 2>
                     : (const void*)bt::bt_persistent_kernel<double, 2>;
}
