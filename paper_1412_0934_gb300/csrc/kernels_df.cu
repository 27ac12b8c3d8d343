// Kernels of the PolDF precision policy (see hydro_device.cuh).
#include "kernels_impl.cuh"

namespace hydro {
const KernelOps& ops_df() { return make_ops<PolDF>(); }
}  // namespace hydro
