// Launch interface of the table-driven forward kernel.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "slos_kernels.cuh"

namespace slos {

struct TabArgs {
    const int32_t *rowptr;    // [F_k + 1]
    const uint32_t *entries;  // CSR parent entries of layer k
    const float *w;           // final layer: prod t! / prod s!  [F_n]
    const int32_t *pat;       // final layer, threshold: pattern index [F_n]
};

cudaError_t slos_tab_init();
// gpw: instance groups served by one warp (1 or 2)
cudaError_t slos_launch_fwd_tab(const FwdArgs &a, const TabArgs &t, int epi, bool save, int blocks_x, int gpw,
                                cudaStream_t s);

}  // namespace slos
