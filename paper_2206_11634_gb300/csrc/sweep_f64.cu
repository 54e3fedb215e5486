// Kernel instantiations for double population storage.
#include "launch_impl.cuh"

namespace lbmmb {
LBMMB_INSTANTIATE(double)
}  // namespace lbmmb
