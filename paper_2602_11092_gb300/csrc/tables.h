// Transition graph of a plan (Sec. II-A.3: the k -> k+1 transitions depend
// only on the input state, so they are built once and reused for every batch
// of unitaries; only the U coefficients change per call).
//
// For layer k (k photons, built for k = 1..n):
//   forward:  fixed-width parent lists (ELL).  State c owns slots
//             ell[c * kw .. c * kw + kw - 1], kw = min(m, k) rounded up to a
//             multiple of 4; slot = (parent rank << 5) | mode, or 0xFFFFFFFF
//             when empty.  (The CSR form with rowptr/entries is what
//             slos_host_transition_table exports; the device keeps the ELL.)
//   backward: dense child table ctab[c'][j] = rank_k(t' + e_j) for every
//             parent c' of layer k-1 and every mode j.
// For the final layer n: w[t] = prod t_j! / prod s_i! and, for threshold
// detection, pat[t] = index of the occupied-mode pattern of t.
#pragma once
#include <stdint.h>

#include <vector>

namespace slos {

struct LayerTables {
    uint32_t *ell = nullptr;     // [F_k * kw]
    int kw = 0;
    int32_t *ctab = nullptr;     // [F_{k-1} * m]
};

constexpr uint32_t kEllEmpty = 0xFFFFFFFFu;

struct PlanTables {
    bool enabled = false;
    std::vector<LayerTables> layer;  // [0..n], layer[0] unused
    float *w = nullptr;              // [F_n]
    int32_t *pat = nullptr;          // [F_n] (threshold only)
    size_t bytes = 0;
};

constexpr size_t kTableBudgetBytes = size_t(1) << 30;  // per plan
constexpr int64_t kMaxTableParent = int64_t(1) << 26;

}  // namespace slos
