// Kernel instantiations for __nv_bfloat16 population storage.
#include "launch_impl.cuh"

namespace lbmmb {
LBMMB_INSTANTIATE(__nv_bfloat16)
}  // namespace lbmmb
