// Head/tail split of the Fock lattice (the transition graph of Sec. II-A.3,
// regrouped so that most of its edges become block-to-block copies).
//
// Split the m modes into the head modes 0..h-1 and the tail modes h..m-1.  A
// composition t of k photons is (t_H, t_L); in descending lexicographic
// order all states with the same head t_H are consecutive, so layer k is a
// sequence of head blocks, one per head composition with |t_H| = r <= k, each
// holding the F(m-h, k-r) tail compositions in their own descending-lex order:
//      rank_k(t) = base_k(t_H) + rank(t_L).
// The parent of t through a head mode j (t_j > 0) is (t_H - e_j, t_L): it sits
// in the head block t_H - e_j of layer k-1, whose tail lattice is the same
// F(m-h, k-r), at the same local position.  So for a whole head block the
// head-mode parents are a fixed set of (parent block base, mode) pairs, one
// per occupied head mode, and U[j, c_k] is the same for every state of the
// block.  Only the tail modes need per-state slots, and those come from one
// small table per tail photon number shared by all head blocks.  In the
// backward direction every parent has all m children: through head mode j the
// child (t_H + e_j, t_L) at the same local position of block t_H + e_j, and
// through tail mode j the child (t_H, t_L + e_j) of block t_H, whose local
// position comes from the shared tail child table.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace slos {

constexpr int kSplitMaxHead = 8;      // head modes per plan (bounds the per-block dispatch)
constexpr int kSplitMaxTail = 8;      // tail modes per plan (one 16-byte child row)
constexpr int kSplitRun = 4;         // consecutive states per warp work item
constexpr int kSplitTile = 32;       // forward: states per CTA output tile (kSplitFwdWarps runs)
constexpr int kSplitMaxTailStates = 65535;  // tail positions are 16-bit in the child rows

// Host-built tables of one layer k >= 2 (all ranks are global ranks within
// their layer).
struct SplitLayerHost {
    // forward: head blocks of layer k in rank order
    //   x = base in layer k, y = size, z = base of block t_H in layer k-1
    //   (the tail parents; 0 when the block has no tail photon), w = rho | qh << 8
    //   with rho = tail photons, qh = occupied head modes
    std::vector<int32_t> fdesc;     // [nblk][4]
    std::vector<uint32_t> fhead;    // [nblk][kSplitMaxHead]: (base of t_H - e_j in layer k-1) << 5 | j
    std::vector<int32_t> fchunk;    // [ceil(F_k / kSplitRun)]: block holding the run's first state
    // backward: head blocks of layer k-1 (the parents)
    //   x = base in layer k-1, y = size, z = base of block t_H in layer k (the
    //   tail children), w = rho (tail photons of the parent)
    std::vector<int32_t> bdesc;     // [nblk][4]
    std::vector<int32_t> bhead;     // [nblk][kSplitMaxHead]: base of t_H + e_j in layer k
    std::vector<int32_t> bchunk;    // [ceil(F_{k-1} / kSplitRun)]
};

// Tail tables over mL = m - h modes, rho = 0..n tail photons.
struct SplitTailHost {
    std::vector<uint32_t> slots;    // rho's rows at soff[rho]: [F(mL, rho)][tw[rho]]
                                    //   (local parent << 5 | h + tail mode, padded with kSlotEmpty)
    std::vector<uint16_t> ctab;     // rho's rows at coff[rho] (rows of 8): local child position of t_L + e_j
    int soff[kMaxPhotons + 1];
    int tw[kMaxPhotons + 1];
    int coff[kMaxPhotons + 1];
};

bool split_eligible(int m, int n, int *h_out);
void split_build_layer_host(int m, int h, int k, SplitLayerHost &out);
void split_build_tail_host(int m, int h, int n, SplitTailHost &out);

struct SplitLayer {
    int nfblk = 0, nbblk = 0;
    int4 *fdesc = nullptr;
    uint32_t *fhead = nullptr;
    int32_t *fchunk = nullptr;
    int4 *bdesc = nullptr;
    int32_t *bhead = nullptr;
    int32_t *bchunk = nullptr;
};

struct SplitTables {
    int h = 0;
    std::vector<SplitLayer> layer;  // [0..n]; layers 2..n filled
    uint32_t *tslots = nullptr;
    uint16_t *tctab = nullptr;
    int soff[kMaxPhotons + 1];
    int tw[kMaxPhotons + 1];
    int coff[kMaxPhotons + 1];
    size_t bytes = 0;
};

struct SplitFwdArgs {
    const float2 *prev;       // a_{k-1}: [NG][Fprev][32]
    float2 *next;             // a_k: [NG][Fk][32] (null for a final layer that keeps nothing)
    const float2 *U;          // [B][m][m]
    void *out;                // final layer: [B][K]
    const float *w;           // final layer: prod t! / prod s!  [F_n]
    const int32_t *pat;       // final layer, threshold: pattern index [F_n]
    const int4 *desc;
    const uint32_t *head;
    const int32_t *chunk;
    const uint32_t *tslots;
    int soff[kMaxPhotons + 1];
    int tw[kMaxPhotons + 1];
    int Fk, Fprev, ntiles;     // ntiles: CTA tiles of kSplitTile states
    int64_t K;
    int m, col, B;
};

struct SplitBwdArgs {
    const float2 *aprev;      // a_{k-1}: [NG][Fprev][32]
    const float2 *Gk;         // G_k (k < n)
    float2 *Gprev;            // G_{k-1}
    const float2 *an;         // a_n (k == n)
    const void *seed;         // see Seed (slos_kernels.cuh)
    const float2 *U;          // [B][m][m]
    float2 *dUpart;           // [NG][gridDim.x][32][m]
    const int4 *desc;
    const int32_t *head;
    const int32_t *chunk;
    const uint16_t *tctab;
    int coff[kMaxPhotons + 1];
    int Fk, Fprev, nruns;      // nruns: warp items of kSplitRun parents
    int m, col, B;
};

// Resident blocks per SM the split kernels' register budgets are sized for.
constexpr int kSplitFwdWarps = kSplitTile / kSplitRun;
#ifndef SLOS_SPLIT_FWD_MINB
#define SLOS_SPLIT_FWD_MINB 3
#endif
constexpr int kSplitFwdMinBlocks = SLOS_SPLIT_FWD_MINB;
constexpr int kSplitBwdWarps = 4;
#ifndef SLOS_SPLIT_BWD_MINB
#define SLOS_SPLIT_BWD_MINB 6
#endif
constexpr int kSplitBwdMinBlocks = SLOS_SPLIT_BWD_MINB;


size_t split_fwd_smem_bytes(int epi);
// The forward layers take the split walk only when this is set (the backward
// layers always do for plans with split tables).
#ifndef SLOS_SPLIT_FWD
#define SLOS_SPLIT_FWD 0
#endif
constexpr bool kSplitForward = SLOS_SPLIT_FWD != 0;

cudaError_t slos_split_init();
cudaError_t slos_launch_fwd_split(const SplitFwdArgs &a, int NG, int epi, bool save, int blocks_x, cudaStream_t s);
cudaError_t slos_launch_bwd_split(const SplitBwdArgs &a, int NG, int seed, int h, int blocks_x, cudaStream_t s);

}  // namespace slos
