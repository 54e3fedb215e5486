// Kernel instantiations for __half population storage.
#include "launch_impl.cuh"

namespace lbmmb {
LBMMB_INSTANTIATE(__half)
}  // namespace lbmmb
