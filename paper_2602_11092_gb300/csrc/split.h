// Head/tail split of the Fock lattice (the transition graph of Sec. II-A.3,
// regrouped so that most of its edges become block-to-block copies), used by
// the backward layers.
//
// Split the m modes into the head modes 0..h-1 and the tail modes h..m-1.  A
// composition t of k photons is (t_H, t_L); in descending lexicographic
// order all states with the same head t_H are consecutive, so layer k is a
// sequence of head blocks, one per head composition with |t_H| = r <= k, each
// holding the F(m-h, k-r) tail compositions in their own descending-lex order:
//      rank_k(t) = base_k(t_H) + rank(t_L).
// Every parent t of layer k-1 has all m children in layer k: through head mode
// j the child (t_H + e_j, t_L), at the same local position of block t_H + e_j
// (whose tail lattice is the same), and through tail mode j the child
// (t_H, t_L + e_j) of block t_H, whose local position comes from one small
// child table per tail photon number shared by all head blocks.  So for a
// whole head block the head children are a fixed set of block offsets, and
// only the tail children need per-state table rows.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace slos {

constexpr int kSplitMaxHead = 8;      // head modes per plan (bounds the per-block dispatch)
constexpr int kSplitMaxTail = 8;      // tail modes per plan (one 16-byte child row)
constexpr int kSplitRun = 4;         // consecutive parents per warp work item
constexpr int kSplitMaxTailStates = 65535;  // tail positions are 16-bit in the child rows

// Host-built tables of one layer k >= 2: the head blocks of layer k-1 (the
// parents), all ranks global within their layer.
struct SplitLayerHost {
    //   x = base in layer k-1, y = size, z = base of block t_H in layer k (the
    //   tail children), w = rho (tail photons of the parent)
    std::vector<int32_t> bdesc;     // [nblk][4]
    std::vector<int32_t> bhead;     // [nblk][kSplitMaxHead]: base of t_H + e_j in layer k
    std::vector<int32_t> bchunk;    // [ceil(F_{k-1} / kSplitRun)]: block holding the run's first parent
};

// Tail child table over mL = m - h modes, rho = 0..n-1 tail photons.
struct SplitTailHost {
    std::vector<uint16_t> ctab;     // rho's rows at coff[rho] (rows of 8): local child position of t_L + e_j
    int coff[kMaxPhotons + 1];
};

bool split_eligible(int m, int n, int *h_out);
void split_build_layer_host(int m, int h, int k, SplitLayerHost &out);
void split_build_tail_host(int m, int h, int n, SplitTailHost &out);

struct SplitLayer {
    int nbblk = 0;
    int4 *bdesc = nullptr;
    int32_t *bhead = nullptr;
    int32_t *bchunk = nullptr;
};

struct SplitTables {
    int h = 0;
    std::vector<SplitLayer> layer;  // [0..n]; layers 2..n filled
    uint16_t *tctab = nullptr;
    int coff[kMaxPhotons + 1];
    size_t bytes = 0;
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
    int *status;               // plan status word (bounds checks of SLOS_DEBUG builds)
    int m, col, B;
    // a_{k-1} recomputed per parent from a_{k-2} instead of read (intermediate
    // layers whose parent layer was not kept): layer k-1's parent slots (rows
    // of 8), a_{k-2} [NG][F_{k-2}][32] and the input mode of photon k-1
    const uint32_t *pslots;
    const float2 *pprev;
    int pcol, Fpp;
};

// Resident blocks per SM the backward kernel's register budget is sized for.
constexpr int kSplitBwdWarps = 4;
// 5 (102 registers): the 16 child loads of a parent are all in flight before
// the tensor-memory batches consume them, which 80 registers (6 blocks) spill
#ifndef SLOS_SPLIT_BWD_MINB
#define SLOS_SPLIT_BWD_MINB 5
#endif
constexpr int kSplitBwdMinBlocks = SLOS_SPLIT_BWD_MINB;

cudaError_t slos_launch_bwd_split(const SplitBwdArgs &a, int NG, int seed, int h, int blocks_x, cudaStream_t s,
                                  bool fuse_prev = false);

}  // namespace slos
