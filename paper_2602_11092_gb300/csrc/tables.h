// Transition graph of a plan (Sec. II-A.3: the k -> k+1 transitions depend
// only on the input state, so they are built once and reused for every batch
// of unitaries; only the U coefficients change per call).
//
// For layer k (k photons, built for k = 1..n):
//   forward:  fixed-width parent slots, kw = min(m, k) rounded up to 4 per
//             state: slot = (parent rank << 5) | mode for every occupied mode
//             of the state, then empty slots (parent 0, mode kMaxModes).
//             Parent ranks are < 2^26.
//   backward: dense child table ctab[c'][j] = rank_k(t' + e_j) for every
//             parent c' of layer k-1 and every mode j.
// For the final layer n: w[t] = prod t_j! / prod s_i!.  Under threshold
// detection the forward walks the final layer in pattern-grouped list order
// (patterns in output order; inside a pattern with support b, the states
// t = 1_b + u in descending-lex order of u), so that the states of a pattern
// are consecutive: layer n's slot rows are stored in that order, with the
// per-position tables of PlanTables.
#pragma once
#include <stdint.h>

#include <vector>

namespace slos {

struct LayerTables {
    uint32_t *slots = nullptr;   // [F_k][kw]
    uint32_t *colinfo = nullptr; // [F_k]: (rank of s - e_c in layer k-1) << 5 | c, c = highest occupied mode of s
    int kw = 0;
    int32_t *ctab = nullptr;     // [F_{k-1} * m]
};

// On-chip forward layout of layer k: the states sorted, stably, by their
// number q of occupied modes, each run of equal q padded to a multiple of 32
// ("positions"); one warp walks a block of 32 positions, all with q parents.
// Block b's rows are slot-major, rows[off + i * 32 + lane] = (parent position
// << 5) | mode of slot i, with blk[b] = off << 4 | q.  Padding positions name
// parent 0 and the zero row of U.
struct FusedLayer {
    uint32_t *rows = nullptr;
    uint32_t *blk = nullptr;
    int nblk = 0;
    int fpad = 0;   // positions (a multiple of 32)
};

struct PlanTables {
    bool enabled = false;
    std::vector<LayerTables> layer;  // [0..n], layer[0] unused
    std::vector<FusedLayer> fused;   // [0..n] when the on-chip forward is used
    int32_t *fused_id = nullptr;     // final layer: output index of each position, -1 for padding
    float *fused_w = nullptr;        // final layer: weight of each position
    float *w = nullptr;              // [F_n]
    // threshold detection, per list position of the final layer
    int32_t *lrank = nullptr;        // [F_n] Fock rank of the state
    int32_t *lpat = nullptr;         // [F_n] its pattern (output index)
    float *lw = nullptr;             // [F_n] its weight w[t]
    int32_t *lseg = nullptr;         // [nseg + 1] forward work items: runs of whole patterns
    int nseg = 0;
    float *gfact = nullptr;          // [F_n]: sqrt(prod t_j!) of the final states (amplitude encoding)
    uint8_t *occ = nullptr;          // [K][m]: occupation of mode j in output k (photon counts for PNR
                                     // outputs, 0/1 for threshold outcomes)
    size_t bytes = 0;
};

constexpr size_t kTableBudgetBytes = size_t(1) << 30;  // per plan
constexpr int64_t kMaxTableParent = int64_t(1) << 26;
constexpr int64_t kMaxEncodeStates = 32768;  // amplitude encoding: the transfer matrix is K x K

}  // namespace slos
