// Launch interface of the table-driven forward kernel.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "slos_kernels.cuh"

namespace slos {

struct TabArgs {
    const uint32_t *ell;      // fixed-width parent lists of layer k [F_k][kw]
    int kw;                   // slots per state, multiple of 4
    const float *w;           // final layer: prod t! / prod s!  [F_n]
    const int32_t *pat;       // final layer, threshold: pattern index [F_n]
};

cudaError_t slos_tab_init();
cudaError_t slos_launch_fwd_tab(const FwdArgs &a, const TabArgs &t, int epi, bool save, int blocks_x, cudaStream_t s);

}  // namespace slos
