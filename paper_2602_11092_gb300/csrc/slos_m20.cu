// Instantiation of the SLOS layer kernels for up to 20 modes.
#include "slos_kernels.cuh"

namespace slos {
SLOS_DEFINE_LAUNCHERS(20)
}  // namespace slos
