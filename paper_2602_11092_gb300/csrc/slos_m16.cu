// Instantiation of the SLOS layer kernels for up to 16 modes.
#include "slos_kernels.cuh"

namespace slos {
SLOS_DEFINE_LAUNCHERS(16)
}  // namespace slos
