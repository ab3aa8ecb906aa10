// Instantiation of the SLOS layer kernels for up to 12 modes.
#include "slos_kernels.cuh"

namespace slos {
SLOS_DEFINE_LAUNCHERS(12)
}  // namespace slos
