// Kernels of the PolF32 precision policy (see hydro_device.cuh).
#include "kernels_impl.cuh"

namespace hydro {
const KernelOps& ops_f32() { return make_ops<PolF32>(); }
}  // namespace hydro
