// Instantiation of the SLOS layer kernels for up to 8 modes.
#include "slos_kernels.cuh"

namespace slos {
SLOS_DEFINE_LAUNCHERS(8)
}  // namespace slos
