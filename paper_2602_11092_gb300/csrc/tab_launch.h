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

// Resident 256-thread blocks per SM the table forward's registers are sized
// for (48 registers); launch grids are sized to fill them.
constexpr int kFwdTabMinBlocks = 5;

cudaError_t slos_tab_init();
cudaError_t slos_launch_fwd_tab(const FwdArgs &a, const TabArgs &t, int epi, bool save, int blocks_x, cudaStream_t s);

}  // namespace slos
