// Launch interface of the table-driven forward kernel (slos_pair.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "slos_kernels.cuh"

namespace slos {

struct TabArgs {
    const uint32_t *slots;    // [F_k][kw] parent slots of layer k
    int kw;                   // slots per state: 4, 8 or 12
    const float *w;           // final layer: prod t! / prod s!  [F_n]
    int *work;                // work-queue counter, zero at launch
    // final layer under threshold detection, walked in list order (tables.h):
    // slots and w are per list position, and
    const int32_t *lrank;     // Fock rank of each position (where a_n is kept)
    const int32_t *lpat;      // pattern of each position
    const int32_t *lseg;      // [nseg + 1] first position of each work item
    int nseg;
};

// Empty slot: parent 0, mode kMaxModes (a zero row of the staged U).
constexpr uint32_t kSlotEmpty = (uint32_t)kMaxModes;
constexpr int slot_width(int m, int k) { return ((m < k ? m : k) + 3) & ~3; }

// Two instance groups per warp, one chunk of consecutive states per warp
// work item, U[j, c_k] in tensor memory.
cudaError_t slos_pair_init();
int slos_pair_resident_blocks(int m);
int slos_pair_warps();
int slos_pair_chunk();
cudaError_t slos_launch_fwd_pair(const FwdArgs &a, const TabArgs &t, int epi, bool save, int blocks, cudaStream_t s);

}  // namespace slos
