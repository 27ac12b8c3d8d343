// Kernels of the PolMixed precision policy (see hydro_device.cuh).
#include "kernels_impl.cuh"

namespace hydro {
const KernelOps& ops_mixed() { return make_ops<PolMixed>(); }
}  // namespace hydro
