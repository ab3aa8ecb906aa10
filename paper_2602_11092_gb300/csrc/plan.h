// Host-side plan: Fock-lattice sizes, photon columns, checkpoint schedule and
// workspace layout.  Built once per (m, n, input state, detection); only the
// unitaries change between calls (Sec. II-A.3).
#pragma once

#include <stdint.h>
#include <stddef.h>

#include <string>
#include <vector>

#include "../../include/slos.h"
#include "tables.h"

namespace slos {

constexpr size_t kAlign = 256;
// Work-queue counters in the workspace: forward layer k uses counter k, a
// recomputed layer q counter kCtrRecompute + q, backward layer k counter
// kCtrBackward + k.
constexpr int kCounters = 64;
constexpr int kCtrRecompute = 16;
constexpr int kCtrBackward = 32;

inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int64_t binom_host(int a, int e);

// Host rank/unrank in descending-lex order (same closed form as the device).
int64_t host_rank(int m, const int *t);
void host_unrank(int m, int k, int64_t r, int *t);

struct BatchedPlan;  // uneven batches (batched.cu)
struct SplitTables;  // head/tail split of the lattice (split.h)

struct Layout {
    // byte offsets into the workspace (SIZE_MAX = absent)
    std::vector<size_t> layer;  // [0..n]: where a_k lives (layer[0] unused)
    size_t g[2];                // G ping-pong
    size_t seedT;               // transposed output gradient
    std::vector<size_t> dupart; // [1..n]: dU partials of layer k
    std::vector<int> bwd_blocks;  // [1..n]: blocks_x of the backward launch of layer k
    size_t dpw;                   // shared seed [F_n] floats (aliases seedT)
    size_t dulayer;               // per-layer dU sums [n][NG][32][m] c64
    size_t counters;              // kCounters work-queue counters (zeroed by each forward / backward call)
    size_t total;
};

struct slos_plan_impl;

}  // namespace slos

struct slos_plan_s;
namespace slos {
void batched_destroy(slos_plan_s *p);
}

struct slos_plan_s {
    int kind;  // 0 = single-shape plan, 1 = uneven batch
    int m, n;
    std::vector<int> s;     // input occupations
    std::vector<int> cols;  // c_1 <= ... <= c_n
    slos_detection_t det;
    int space = 0;          // slos_space_t: 0 Fock, 1 collision-free states only
    int64_t K;              // outputs per instance
    std::vector<int64_t> F; // |F(m, k)| for k = 0..n
    float inv_sfact;
    int stride;             // checkpoint stride s (1 = every layer kept)
    std::vector<char> stored;  // [0..n]: layer kept by a saving forward
    int pat_off[16];
    int device;
    int sm_count;
    int *d_status;          // device status word (owned)
    slos::PlanTables tab;   // transition graph (owned; empty when too large)
    int fused_ni = 0;       // instances per CTA of the on-chip inference forward (0: not eligible)
    int fused_threads = 512;    // its CTA size
    int fused_cap[2] = {1, 1};  // its buffer capacities (states per instance, even / odd layers)
    bool fused_sorted = false;  // walks the sorted layout (tab.fused) instead of Fock order
    int prefix_L = 0;           // layers 1..prefix_L run on chip in one launch each way (0: none)
    // launch shapes picked by slos_autotune (negative / zero: the defaults)
    int tune_prefix_L = -1;     // prefix depth: 0 (none) or 2..prefix_L
    int tune_prefix_ni = 0;     // prefix instances per CTA: 1, 2 or 4
    int tune_fwd_bps = 0;       // forward layer grid: blocks per SM (at most the resident count)
    int tune_bwd_bps = 0;       // backward layer grid: blocks per SM (at most the layout's)
    slos::BatchedPlan *batched;
    slos::SplitTables *split = nullptr;  // split-lattice tables (null: slot-table kernels only)
};
