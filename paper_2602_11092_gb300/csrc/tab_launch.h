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
    int *work;                // work-queue counter, zero at launch
    int items_per_group;      // CTA items (kWarpsPerBlock chunks of 32 states) per instance group
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
#ifndef SLOS_FWD_TAB_MINB_STORE
#define SLOS_FWD_TAB_MINB_STORE 6
#endif
#ifndef SLOS_FWD_TAB_MINB_FINAL
#define SLOS_FWD_TAB_MINB_FINAL 6
#endif
constexpr int kFwdTabMinBlocksStore = SLOS_FWD_TAB_MINB_STORE;
constexpr int kFwdTabMinBlocksFinal = SLOS_FWD_TAB_MINB_FINAL;
constexpr int kFwdTabTile = 16;
constexpr int fwd_tab_min_blocks(int epi) { return epi == 0 ? kFwdTabMinBlocksStore : kFwdTabMinBlocksFinal; }
inline int fwd_tab_resident_blocks(int epi) { return fwd_tab_min_blocks(epi); }
// U[j, c_k] from tensor memory instead of shared memory (slos_tab.cu)
#ifndef SLOS_FWD_TMEM_U
#define SLOS_FWD_TMEM_U 1
#endif
constexpr bool kFwdTabTmemU = SLOS_FWD_TMEM_U != 0;
// dynamic shared memory of a table-forward block: per warp a [32][kFwdTabTile + 1] tile
inline size_t fwd_tab_smem_bytes(int epi) {
    const size_t cells = (size_t)kWarpsPerBlock * 32 * (kFwdTabTile + 1);
    return epi == 1 ? cells * sizeof(float) : (epi == 2 ? cells * sizeof(float2) : 0);
}

cudaError_t slos_tab_init();
// Two instance groups per warp (slos_pair.cu): same tables and queue.
#ifndef SLOS_FWD_PAIR
#define SLOS_FWD_PAIR 1
#endif
constexpr bool kFwdPair = SLOS_FWD_PAIR != 0;
cudaError_t slos_pair_init();
int slos_pair_resident_blocks(int m);
int slos_pair_warps();
int slos_pair_chunk();
cudaError_t slos_launch_fwd_pair(const FwdArgs &a, const TabArgs &t, int epi, bool save, int blocks, cudaStream_t s);
cudaError_t slos_launch_fwd_tab(const FwdArgs &a, const TabArgs &t, int epi, bool save, int blocks_x, cudaStream_t s);

}  // namespace slos
