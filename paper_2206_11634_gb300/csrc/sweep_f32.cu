// Kernel instantiations for float population storage.
#include "launch_impl.cuh"

namespace lbmmb {
LBMMB_INSTANTIATE(float)
}  // namespace lbmmb
