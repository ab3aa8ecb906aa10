// Launch interface of the table-driven forward kernel.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "slos_kernels.cuh"

namespace slos {

struct TabArgs {
    const uint32_t *slots;    // [F_k][kw] parent slots of layer k
    int kw;                   // slots per state: 4, 8 or 12
    const float *w;           // final layer: prod t! / prod s!  [F_n]
    const int32_t *pat;       // final layer, threshold: pattern index [F_n]
};

// Empty slot: parent 0, mode kMaxModes (a zero row of the staged U).
constexpr uint32_t kSlotEmpty = (uint32_t)kMaxModes;
constexpr int slot_width(int m, int k) { return ((m < k ? m : k) + 3) & ~3; }

// Resident 256-thread blocks per SM the table forward's registers are sized
// for (48 registers); launch grids are sized to fill them.
constexpr int kFwdTabMinBlocks = 5;

cudaError_t slos_tab_init();
cudaError_t slos_launch_fwd_tab(const FwdArgs &a, const TabArgs &t, int epi, bool save, int blocks_x, cudaStream_t s);

}  // namespace slos
