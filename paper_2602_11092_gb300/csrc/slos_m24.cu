// Instantiation of the SLOS layer kernels for up to 24 modes.
#include "slos_kernels.cuh"

namespace slos {
SLOS_DEFINE_LAUNCHERS(24)
}  // namespace slos
