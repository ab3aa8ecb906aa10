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
// for; launch grids are sized to fill them.  Measured on the m=16, n=8
// training step: the final layer runs fastest at 8 blocks (32 registers, 64
// warps per SM, which its output tile of kFwdTabTile states per warp leaves
// room for), the intermediate layers at 5 (48 registers: at 32 they lose more
// to the smaller register budget than they gain from the warps).
constexpr int kFwdTabMinBlocksStore = 5;
constexpr int kFwdTabMinBlocksFinal = 8;
constexpr int kFwdTabTile = 16;
constexpr int fwd_tab_min_blocks(int epi) { return epi == 0 ? kFwdTabMinBlocksStore : kFwdTabMinBlocksFinal; }
// The same walk with U in tensor memory (slos_fwd_tabu_kernel): one 64-column
// allocation per CTA, so at most 8 resident CTAs per SM.
#ifndef SLOS_FWD_TMEM_U
#define SLOS_FWD_TMEM_U 1
#endif
#ifndef SLOS_FWD_TABU_MINB_STORE
#define SLOS_FWD_TABU_MINB_STORE 6
#endif
#ifndef SLOS_FWD_TABU_MINB_FINAL
#define SLOS_FWD_TABU_MINB_FINAL 6
#endif
constexpr bool kFwdTabTmemU = SLOS_FWD_TMEM_U != 0;
constexpr int fwd_tabu_min_blocks(int epi) { return epi == 0 ? SLOS_FWD_TABU_MINB_STORE : SLOS_FWD_TABU_MINB_FINAL; }
inline int fwd_tab_resident_blocks(int epi) { return kFwdTabTmemU ? fwd_tabu_min_blocks(epi) : fwd_tab_min_blocks(epi); }
// dynamic shared memory of a table-forward block: per warp a [32][kFwdTabTile + 1] tile
inline size_t fwd_tab_smem_bytes(int epi) {
    const size_t cells = (size_t)kWarpsPerBlock * 32 * (kFwdTabTile + 1);
    return epi == 1 ? cells * sizeof(float) : (epi == 2 ? cells * sizeof(float2) : 0);
}

cudaError_t slos_tab_init();
cudaError_t slos_launch_fwd_tab(const FwdArgs &a, const TabArgs &t, int epi, bool save, int blocks_x, cudaStream_t s);

}  // namespace slos
