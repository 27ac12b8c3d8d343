// Kernels of the PolF64 precision policy (see hydro_device.cuh).
#include "kernels_impl.cuh"

namespace hydro {
const KernelOps& ops_f64() { return make_ops<PolF64>(); }
}  // namespace hydro
