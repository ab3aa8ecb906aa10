// Uneven batches: instances of different (m, n, input, detection) in ONE
// persistent kernel launch (graph-capturable), with launch shapes picked by
// an autotuner.
//
// Instances with the same shape are packed 16 per "lane group", a shape's
// remaining instances in groups of 8 and 4 (9..12 left: 8 + 4); a warp serves one lane group
// and walks 32 / width Fock states at a time (part p of the warp takes every
// (32 / width)-th state, lane % width is the instance), so the ~14 instances
// a shape typically has in a 1024-instance batch fill most lanes and a shape
// with a few instances does not walk idle lanes' rows.  Layer k of a lane
// group lives in workspace as complex64 [F_k][width].  Each shape's
// transition graph is built once on the GPU at plan time as parent slots:
// slot = (parent position << 5) | j for every mode j with t_j > 0, padded
// with a slot that reads a zero row of U (Sec. II-A.3: the transitions
// depend only on the input state).  A state with q occupied modes has q
// parents, so each layer (but a PNR output layer, kept in Fock order for
// the output) is stored with its states sorted, stably, by q rounded up to
// even: a section of rows 2, 4, ..., 12 slots wide, so that no state pays
// for the widest one.  A layer's "position" of a state is its place in that
// order; the next layer's slots use positions.  Under threshold detection
// the final layer's positions are its pattern-grouped list order instead
// (patterns in output order, a pattern's states consecutive; it agrees with
// the sections, since the patterns come by increasing |b|), and a work item
// of that layer is a run of whole patterns, so one warp sums each pattern in
// a fixed order and stores it once.  A final state's weight
// prod t_j! / prod s_i! is a per-position table built with the slots.
// Work item = (lane group, layer k, chunk of consecutive Fock states).  Items are listed layer by
// layer (all layer-1 items of every lane group, then all layer-2 items, ...),
// largest lane groups first inside a layer (longest-processing-time order).
// Warps pop items in that order with one atomic counter; an item of layer
// k >= 2 waits until every item of its lane group's layer k-1 has finished
// (a per-descriptor completion counter).  Every item an item waits on was
// popped earlier by a warp that is running, so the wait always ends; it is
// bounded anyway, and a wait that runs out records SLOS_ERR_TIMEOUT and the
// item id in the plan's status word and stops the warp.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/slos.h"
#include "common.cuh"
#include "plan.h"
#include "profile.h"

namespace slos {
slos_status_t fail(slos_status_t st, const std::string &msg);

constexpr int kBMax = 20;   // modes handled by the persistent kernel (m <= 20)
constexpr int kBLanes = 16; // instances per lane group
constexpr uint32_t kSlotEmpty = (uint32_t)kBMax;   // parent 0, mode kBMax (a zero row of U)
constexpr int64_t kBMaxParent = int64_t(1) << 27;  // parent ranks in 27 bits
constexpr int kBSec = 12;   // one section per occupied-mode count 1..12
// slot-row width of section s (q = s + 1 occupied modes): q rounded up to even
__host__ __device__ constexpr int sec_width(int s) { return (s + 2) & ~1; }

struct BShape {
    int m, n, det, K;
    int cols[kMaxPhotons];
    int64_t F[kMaxPhotons + 1];
    int64_t slot_off[kMaxPhotons + 1];  // element offset of layer k's slots in the table buffer
    int64_t w_off;                      // final-layer weights prod t! / prod s! (float) [F_n]
    int kw[kMaxPhotons + 1];            // widest slot row of layer k (even, <= 12)
    // Layer k is stored in sections of states with q = s + 1 occupied modes
    // (s = 0 .. kBSec-1), each section with rows of sec_width(s) slots (q
    // rounded up to even, for aligned vector loads; a walk reads q of them);
    // positions sec_pos[k][s] .. sec_pos[k][s+1]-1, rows from element
    // sec_off[k][s] of the layer's table.  An unsorted layer is one section,
    // s = kw - 1 (rows of kw slots, all of them walked).
    int sec_pos[kMaxPhotons + 1][kBSec + 1];
    int64_t sec_off[kMaxPhotons + 1][kBSec];
    float inv_sfact;
    int nclass;                         // threshold: pattern classes j = 1 .. min(n, m)
    int pat_off[kMaxPhotons + 2];       // first pattern index with j occupied modes
    int pat_cnt[kMaxPhotons + 2];       // final states per pattern with j occupied modes: C(n-1, j-1)
    int64_t pat_base[kMaxPhotons + 2];  // first position of class j in the grouped list
};

struct BLaneGroup {
    int shape;
    int width;            // instances per lane group: 16, 8 or 4 (a shape's remainder after the 16s)
    int inst[kBLanes];    // global instance index per lane, -1 = empty lane
    int64_t buf[2];       // workspace byte offsets of the two layer buffers
};

struct BDesc {
    int lg;      // lane group
    int k;       // layer
    int dep;     // descriptor of layer k-1 of the same lane group (-1 for k = 1)
    int nchunks;
};

struct BArgs {
    const BShape *shapes;
    const BLaneGroup *lgs;
    const BDesc *desc;
    const int64_t *first_item;  // [ndesc + 1]
    const uint32_t *slots;      // all shapes' tables
    int ndesc;
    int64_t total_items;
    int chunk;
    const float2 *U;
    const int64_t *u_off;
    float *out;
    const int64_t *out_off;
    char *ws;
    int *done;          // [ndesc] completion counters (zeroed per launch)
    unsigned long long *head;  // work counter (zeroed per launch)
    int *status;        // plan status word
    long long spin_limit;
};

// Occupied modes of state c of layer k (descending-lex rank, bar unranking
// of common.cuh) and the section it goes to: q - 1.
template <int MMAX>
__device__ __forceinline__ int state_section(const BShape &sh, int k, int64_t c) {
    const int m = sh.m, L = k + m - 1;
    int p[MMAX];
    unrank_bars<MMAX>(c, m, L, p);
    int q = 0;
#pragma unroll
    for (int j = 0; j < MMAX; ++j)
        if (j < m && occupation<MMAX>(j, m, L, p) > 0) ++q;
    return q - 1;
}

// Stable partition of layer k by section, in two passes over blocks of 256
// consecutive states: (1) cnt[blk][s] = states of block blk in section s;
// (2) pos[c] = base[blk][s] + rank of c among the block's states of its
// section, base being the section start plus the counts of earlier blocks
// (an exclusive scan the host does between the passes).
template <int MMAX>
__global__ void __launch_bounds__(256) section_pass_kernel(const BShape sh, int k, int *cnt, const int *base,
                                                            int *pos) {
    __shared__ int wcnt[8][kBSec];
    const int64_t c = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int sec = c < sh.F[k] ? state_section<MMAX>(sh, k, c) : -1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int wrank = 0;
#pragma unroll
    for (int q = 0; q < kBSec; ++q) {
        const unsigned bal = __ballot_sync(0xffffffffu, sec == q);
        if (sec == q) wrank = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) wcnt[warp][q] = __popc(bal);
    }
    __syncthreads();
    if (!pos) {
        if (threadIdx.x < kBSec) {
            int t = 0;
            for (int w = 0; w < 8; ++w) t += wcnt[w][threadIdx.x];
            cnt[(size_t)blockIdx.x * kBSec + threadIdx.x] = t;
        }
        return;
    }
    if (sec < 0) return;
    int r = wrank;
    for (int w = 0; w < warp; ++w) r += wcnt[w][sec];
    pos[c] = base[(size_t)blockIdx.x * kBSec + sec] + r;
}

// Tables of layer k of one shape, one thread per state, with the index
// arithmetic of the single-shape kernels (common.cuh): the row of state c
// (at position cpos[c], or c in an unsorted layer) holds
//   (position of t - e_j in layer k-1 << 5) | j
// for the occupied modes j of t in mode order, then padding; ppos maps the
// parent layer's ranks to positions (null: unsorted).  For the final layer
// also w[position] = prod t_j! / prod s_i!.  With `listed` (the final layer
// of a threshold shape) the position is the state's place in the
// pattern-grouped list: patterns in output order (|b|, then colex), and
// inside a pattern the states t with support b in descending-lex order of
// t - 1_b, a composition of n - |b| photons over |b| modes, ranked with the
// same bar formula.
template <int MMAX>
__global__ void build_slots_kernel(const BShape sh, int k, uint32_t *tab, const int *ppos, const int *cpos,
                                   float *w, bool listed) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= sh.F[k]) return;
    const int m = sh.m;
    const int L = k + m - 1;
    int p[MMAX];
    unrank_bars<MMAX>(c, m, L, p);
    int64_t S = 0;
    int q = 0;
    float fprod = 1.f;
    uint32_t supp = 0;
    int tb[MMAX];  // occupations of the occupied modes, in mode order
    uint32_t e[MMAX];
#pragma unroll
    for (int j = 0; j < MMAX; ++j) {
        if (j < m) {
            const int tj = occupation<MMAX>(j, m, L, p);
            if (tj > 0) {
                tb[q] = tj;
                int64_t r = c - S;
                if (ppos) r = ppos[r];
                e[q++] = ((uint32_t)r << 5) | (uint32_t)j;
                fprod *= c_fact.v[tj];
                supp |= 1u << j;
            }
            if (j < m - 1) S += (int64_t)binom_m1(p[j], m - 2 - j);
        }
    }
    const int nb = q;
    int64_t at = c;
    if (listed) {
        const int np = k - nb, Lp = np + nb - 1;
        int64_t r = 0;
        int cum = 0;
        for (int b = 0; b + 1 < nb; ++b) {
            cum += tb[b] - 1;
            r += (int64_t)binom(Lp - 1 - b - cum, nb - 1 - b);
        }
        at = sh.pat_base[nb] + (int64_t)colex_rank(supp) * sh.pat_cnt[nb] + r;
    } else if (cpos) {
        at = cpos[c];
    }
    uint32_t *dst;
    int width;
    if (cpos || listed) {
        const int sec = nb - 1;
        width = sec_width(sec);
        dst = tab + sh.sec_off[k][sec] + (at - sh.sec_pos[k][sec]) * width;
    } else {
        width = sh.kw[k];
        dst = tab + c * width;
    }
    for (int i = 0; i < nb; ++i) dst[i] = e[i];
    for (int i = nb; i < width; ++i) dst[i] = kSlotEmpty;
    if (w) w[at] = fprod * sh.inv_sfact;
}

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Slot rows of up to kBStage consecutive positions are staged per warp in
// shared memory by one coalesced warp-wide copy, so a walk step waits for
// one global round trip (its parent rows) instead of two (slot row, then
// parent rows).
constexpr int kBStage = 32;
constexpr int kBSlotWords = kBStage * 12;                     // widest rows: 12 slots
constexpr int kBWarpF2 = (kBMax + 1) * kBLanes + kBSlotWords;  // per warp: U column, two staging buffers (float2 units)

__device__ __forceinline__ void b_cp4(uint32_t *dst, const uint32_t *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
template <int N>
__device__ __forceinline__ void b_cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// The slot rows of positions [start, start + n) into dst, as one cp.async group.
__device__ __forceinline__ void stage_issue(const uint32_t *__restrict__ tab, int pos0, int KW, int start, int n,
                                            uint32_t *dst, int lane) {
    const uint32_t *src = tab + (size_t)(start - pos0) * KW;
    for (int i = lane; i < n * KW; i += 32) b_cp4(dst + i, src + i);
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Walk of nwin windows of consecutive positions (win(i, start, n) gives window
// i), each one's slot rows staged in one of the warp's two buffers while the
// previous window is walked: proc(i, start, n, rows) runs once the rows are in.
template <typename Win, typename Proc>
__device__ __forceinline__ void staged_walk(int nwin, Win win, Proc proc, const uint32_t *__restrict__ tab, int pos0,
                                            int KW, uint32_t *sbuf, int lane) {
    if (nwin <= 0) return;
    int s0, n0;
    win(0, s0, n0);
    __syncwarp();
    stage_issue(tab, pos0, KW, s0, n0, sbuf, lane);
    for (int i = 0; i < nwin; ++i) {
        int s, n;
        win(i, s, n);
        if (i + 1 < nwin) {
            int s1, n1;
            win(i + 1, s1, n1);
            stage_issue(tab, pos0, KW, s1, n1, sbuf + ((i + 1) & 1) * kBSlotWords, lane);
            b_cp_wait<1>();
        } else {
            b_cp_wait<0>();
        }
        __syncwarp();  // every lane's copies of window i are in
        proc(i, s, n, sbuf + (i & 1) * kBSlotWords);
        __syncwarp();  // window i read before its buffer takes window i + 2
    }
}

// Amplitude of one state from its staged slot row srow (KW slots, the first
// QV of them occupied) for the lane's instance.  us: this warp's staged
// column of U, row j = U[j][col] per lane (row kBMax zero); prev: layer k-1
// of this lane (rows of LW complex64).  Parent rows are plain (L1-cached)
// loads: the wait on layer k-1's completion counter has ordered them after
// its writes.
template <int KW, int QV, int LW>
__device__ __forceinline__ float2 b_state_amp(const uint32_t *srow, const float2 *us, const char *prev,
                                              bool first_layer) {
    uint32_t e[KW];
    const uint2 *s2 = reinterpret_cast<const uint2 *>(srow);  // rows of an even number of slots: 8-byte aligned
#pragma unroll
    for (int q2 = 0; q2 < KW / 2; ++q2) {
        const uint2 w2 = s2[q2];
        e[2 * q2] = w2.x;
        e[2 * q2 + 1] = w2.y;
    }
    if (first_layer) return us[(e[0] & 31u) * kBLanes];  // one photon: a_1(e_j) = U[j][col]
    float2 v[QV];
    // parent position (e >> 5) times the row of LW complex64
#pragma unroll
    for (int q = 0; q < QV; ++q)
        v[q] = *reinterpret_cast<const float2 *>(prev + (size_t)(e[q] & ~31u) * (LW / 4));
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < QV; ++q) acc = cfma(us[(e[q] & 31u) * kBLanes], v[q], acc);
    return acc;
}

// Positions c0 + part, c0 + part + P, ... < c1 of one section (P = 32 / LW
// parts of the warp, lane il of each part = instance il of the lane group):
// the next layer's amplitudes, or the PNR output probabilities (Fock order).
// Windows of kBStage positions (a multiple of P, so each part keeps its
// positions).
template <int KW, int QV, int LW>
__device__ __forceinline__ void fwd_states(const uint32_t *__restrict__ tab, int pos0, int c0, int c1, int part,
                                           int lane, uint32_t *sbuf, const float2 *us, const char *prev,
                                           bool first_layer, bool last, float2 *next, float *outp,
                                           const float *__restrict__ wtab) {
    constexpr int P = 32 / LW;
    // positions fit in 32 bits (at most C(31, 12) < 2^28 per layer)
    staged_walk(
        (c1 - c0 + kBStage - 1) / kBStage,
        [&](int i, int &st, int &nb) {
            st = c0 + i * kBStage;
            nb = min(kBStage, c1 - st);
        },
        [&](int, int cb, int nb, const uint32_t *rows) {
            for (int c = cb + part; c < cb + nb; c += P) {
                const float2 acc = b_state_amp<KW, QV, LW>(rows + (c - cb) * KW, us, prev, first_layer);
                if (!last) next[(uint32_t)c * LW] = acc;
                else if (outp) outp[c] = __ldg(wtab + c) * (acc.x * acc.x + acc.y * acc.y);
            }
        },
        tab, pos0, KW, sbuf, lane);
}

// Threshold detection, final layer in list order: patterns [P0, P1) of
// class j (cnt states each, the first at list position base), whose output
// indices start at pat_first.  Each pattern's probability is one sum in
// list order: with one state per pattern the parts of the warp take
// patterns in turn; otherwise they take the states of each pattern in turn
// (part p: states p, p + P, ... of the pattern) and add their partial sums
// (lanes il, il + LW, ... in a fixed order).  The sum does not depend on the
// launch shape or on how the slot rows are staged: windows of whole patterns
// (cnt <= kBStage) or, for larger patterns, pieces of kBStage states, which
// keep each part's states and their order.
template <int KW, int QV, int LW>
__device__ __forceinline__ void thresh_patterns(const uint32_t *__restrict__ tab, int pos0, int64_t base, int cnt,
                                                int64_t P0, int64_t P1, int pat_first, int part, int lane,
                                                uint32_t *sbuf, const float2 *us, const char *prev, bool first_layer,
                                                float *outp, const float *__restrict__ wtab) {
    constexpr int P = 32 / LW;
    auto combine_store = [&](float sum, int64_t Q) {
        if (P == 8) sum += __shfl_xor_sync(0xffffffffu, sum, 4);
        if (P >= 4) sum += __shfl_xor_sync(0xffffffffu, sum, 8);
        sum += __shfl_xor_sync(0xffffffffu, sum, 16);
        if (part == 0 && outp) outp[pat_first + Q] = sum;
    };
    if (cnt == 1) {
        const int q0 = (int)(base + P0), q1 = (int)(base + P1);
        staged_walk(
            (q1 - q0 + kBStage - 1) / kBStage,
            [&](int i, int &st, int &nb) {
                st = q0 + i * kBStage;
                nb = min(kBStage, q1 - st);
            },
            [&](int, int cb, int nb, const uint32_t *rows) {
                for (int c = cb + part; c < cb + nb; c += P) {
                    const float2 acc = b_state_amp<KW, QV, LW>(rows + (c - cb) * KW, us, prev, first_layer);
                    if (outp) outp[pat_first + (c - base)] = __ldg(wtab + c) * (acc.x * acc.x + acc.y * acc.y);
                }
            },
            tab, pos0, KW, sbuf, lane);
        return;
    }
    if (cnt <= kBStage) {
        const int per = kBStage / cnt;  // whole patterns per window
        staged_walk(
            (int)((P1 - P0 + per - 1) / per),
            [&](int i, int &st, int &nb) {
                const int64_t Qw = P0 + (int64_t)i * per;
                st = (int)(base + Qw * cnt);
                nb = (int)min((int64_t)per, P1 - Qw) * cnt;
            },
            [&](int i, int cw, int nb, const uint32_t *rows) {
                const int64_t Qw = P0 + (int64_t)i * per;
                for (int64_t Q = Qw; Q < Qw + nb / cnt; ++Q) {
                    const int c0 = (int)(base + Q * cnt);
                    float sum = 0.f;
                    for (int c = c0 + part; c < c0 + cnt; c += P) {
                        const float2 acc = b_state_amp<KW, QV, LW>(rows + (c - cw) * KW, us, prev, first_layer);
                        sum += __ldg(wtab + c) * (acc.x * acc.x + acc.y * acc.y);
                    }
                    combine_store(sum, Q);
                }
            },
            tab, pos0, KW, sbuf, lane);
        return;
    }
    const int npc = (cnt + kBStage - 1) / kBStage;  // pieces per pattern
    float sum = 0.f;
    staged_walk(
        (int)(P1 - P0) * npc,
        [&](int i, int &st, int &nb) {
            const int64_t Q = P0 + i / npc;
            const int piece = (i % npc) * kBStage;
            st = (int)(base + Q * cnt) + piece;
            nb = min(kBStage, cnt - piece);
        },
        [&](int i, int cs, int nb, const uint32_t *rows) {
            if (i % npc == 0) sum = 0.f;
            for (int c = cs + part; c < cs + nb; c += P) {
                const float2 acc = b_state_amp<KW, QV, LW>(rows + (c - cs) * KW, us, prev, first_layer);
                sum += __ldg(wtab + c) * (acc.x * acc.x + acc.y * acc.y);
            }
            if (i % npc == npc - 1) combine_store(sum, P0 + i / npc);
        },
        tab, pos0, KW, sbuf, lane);
}

// Work items of class j of a threshold final layer: runs of whole patterns
// of about `chunk` states.
__host__ __device__ __forceinline__ int64_t thresh_per_item(const BShape &sh, int j, int chunk) {
    const int64_t per = chunk / sh.pat_cnt[j];
    return per > 0 ? per : 1;
}
__host__ __device__ __forceinline__ int64_t thresh_items(const BShape &sh, int j, int chunk) {
    const int64_t npat = sh.pat_off[j + 1] - sh.pat_off[j];
    return (npat + thresh_per_item(sh, j, chunk) - 1) / thresh_per_item(sh, j, chunk);
}

// One work item of lane group g (LW = its width: 16 or 8 instances): layer
// k's positions of the item's section, or (threshold final layer) its run of
// whole patterns.  The warp's 32 / LW parts take positions in turn; lane il
// of each part is instance il of the lane group.
template <int LW>
__device__ __forceinline__ void b_item(const BArgs &a, const BLaneGroup &g, const BShape &sh, int k, int64_t chunk_id,
                                       int lane, float2 *us, uint32_t *sbuf) {
    constexpr int P = 32 / LW;
    const int part = lane / LW, il = lane % LW;
    const int n = sh.n;
    const int inst = g.inst[il];
    const bool valid = inst >= 0;
    float *outp = valid ? a.out + a.out_off[inst] : nullptr;
    const int m = sh.m;
    const int col = sh.cols[k - 1];
    __syncwarp();
    for (int j = part; j < m; j += P)
        us[j * kBLanes + il] = valid ? a.U[a.u_off[inst] + (int64_t)j * m + col] : make_float2(0.f, 0.f);
    __syncwarp();
    const char *prev = a.ws + g.buf[(n - 1 - (k - 1)) & 1] + il * sizeof(float2);
    const uint32_t *tab = a.slots + sh.slot_off[k];
    const float *wtab = reinterpret_cast<const float *>(a.slots + sh.w_off);
    const float2 *usl = us + il;
    if (k == n && sh.det == SLOS_DETECT_THRESHOLD) {
        // the item's class and run of patterns (items counted class by class)
        int j = 1;
        int64_t rem = chunk_id;
        for (; j < sh.nclass; ++j) {
            const int64_t nit = thresh_items(sh, j, a.chunk);
            if (rem < nit) break;
            rem -= nit;
        }
        const int64_t per = thresh_per_item(sh, j, a.chunk);
        const int64_t P0 = rem * per;
        const int64_t P1 = min(P0 + per, (int64_t)(sh.pat_off[j + 1] - sh.pat_off[j]));
        const int sec = j - 1;
        const int p0 = sh.sec_pos[k][sec];
        const uint32_t *st = tab + sh.sec_off[k][sec];
#define SLOS_B_THR(W, Q)                                                                                         \
    thresh_patterns<W, Q, LW>(st, p0, sh.pat_base[j], sh.pat_cnt[j], P0, P1, sh.pat_off[j], part, lane, sbuf, usl, \
                              prev, k == 1, outp, wtab)
        switch (sec) {
            case 0: SLOS_B_THR(2, 1); break;
            case 1: SLOS_B_THR(2, 2); break;
            case 2: SLOS_B_THR(4, 3); break;
            case 3: SLOS_B_THR(4, 4); break;
            case 4: SLOS_B_THR(6, 5); break;
            case 5: SLOS_B_THR(6, 6); break;
            case 6: SLOS_B_THR(8, 7); break;
            case 7: SLOS_B_THR(8, 8); break;
            case 8: SLOS_B_THR(10, 9); break;
            case 9: SLOS_B_THR(10, 10); break;
            case 10: SLOS_B_THR(12, 11); break;
            default: SLOS_B_THR(12, 12); break;
        }
#undef SLOS_B_THR
    } else {
        // the item's section: chunks are counted section by section, so no
        // item straddles two widths
        int sec = 0;
        int64_t rem = chunk_id;
        for (; sec < kBSec - 1; ++sec) {
            const int64_t nch = (sh.sec_pos[k][sec + 1] - sh.sec_pos[k][sec] + a.chunk - 1) / a.chunk;
            if (rem < nch) break;
            rem -= nch;
        }
        const int p0 = sh.sec_pos[k][sec];
        const int c0 = p0 + (int)rem * a.chunk;
        const int c1 = min(c0 + a.chunk, sh.sec_pos[k][sec + 1]);
        float2 *next = reinterpret_cast<float2 *>(a.ws + g.buf[(n - 1 - k) & 1]) + il;
        const uint32_t *st = tab + sh.sec_off[k][sec];
#define SLOS_B_SEC(W, Q) \
    fwd_states<W, Q, LW>(st, p0, c0, c1, part, lane, sbuf, usl, prev, k == 1, k == n, next, outp, wtab)
        switch (sec) {
            case 0: SLOS_B_SEC(2, 1); break;
            case 1: SLOS_B_SEC(2, 2); break;
            case 2: SLOS_B_SEC(4, 3); break;
            case 3: SLOS_B_SEC(4, 4); break;
            case 4: SLOS_B_SEC(6, 5); break;
            case 5: SLOS_B_SEC(6, 6); break;
            case 6: SLOS_B_SEC(8, 7); break;
            case 7: SLOS_B_SEC(8, 8); break;
            case 8: SLOS_B_SEC(10, 9); break;
            case 9: SLOS_B_SEC(10, 10); break;
            case 10: SLOS_B_SEC(12, 11); break;
            default: SLOS_B_SEC(12, 12); break;
        }
#undef SLOS_B_SEC
    }
}

// MINB: resident 256-thread blocks per SM the register allocation is sized for
// (a tuning dimension: fewer registers, more warps in flight).
template <int MINB>
__global__ void __launch_bounds__(256, MINB) slos_batched_kernel(BArgs a) {
    extern __shared__ float2 us_all[];  // per warp: U column [kBMax + 1][16], then kBSlotWords staged slots
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float2 *us = us_all + warp * kBWarpF2;
    uint32_t *sbuf = reinterpret_cast<uint32_t *>(us + (kBMax + 1) * kBLanes);
    if (lane < kBLanes) us[kBMax * kBLanes + lane] = make_float2(0.f, 0.f);
    int lo = 0;  // descriptor of the previous item: items are handed out in increasing order
    for (;;) {
        unsigned long long q = 0;
        if (lane == 0) q = atomicAdd(a.head, 1ull);
        q = __shfl_sync(0xffffffffu, q, 0);
        if ((int64_t)q >= a.total_items) break;
        // descriptor of item q: last i >= lo with first_item[i] <= q
        if (lo + 1 < a.ndesc && a.first_item[lo + 1] <= (int64_t)q) {
            int hi = a.ndesc - 1;
            ++lo;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (a.first_item[mid] <= (int64_t)q) lo = mid;
                else hi = mid - 1;
            }
        }
        const BDesc d = a.desc[lo];
        const int64_t chunk_id = (int64_t)q - a.first_item[lo];
        const BLaneGroup &g = a.lgs[d.lg];
        const BShape &sh = a.shapes[g.shape];
        const int k = d.k;
        if (d.dep >= 0) {
            const int need = a.desc[d.dep].nchunks;
            long long spins = 0;
            bool ok = true;
            if (lane == 0) {
                while (ld_acquire(a.done + d.dep) < need) {
                    if (++spins > a.spin_limit) {
                        ok = false;
                        break;
                    }
                    __nanosleep(200);
                }
                if (!ok) {
                    atomicCAS(a.status, 0, (int)SLOS_ERR_TIMEOUT);
                    atomicExch(a.status + 1, (int)q);
                }
            }
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) return;
            __syncwarp();
            __threadfence();
        }
        if (g.width == 4) b_item<4>(a, g, sh, k, chunk_id, lane, us, sbuf);
        else if (g.width == 8) b_item<8>(a, g, sh, k, chunk_id, lane, us, sbuf);
        else b_item<16>(a, g, sh, k, chunk_id, lane, us, sbuf);
        __threadfence();
        __syncwarp();
        if (lane == 0) atomicAdd(a.done + lo, 1);
    }
}

// Layers stored sorted by occupied modes: all but layer 1 (one section
// anyway) and a PNR output layer (written in Fock order).
static bool layer_sorted(const BShape &sh, int k) { return k >= 2 && !(k == sh.n && sh.det == SLOS_DETECT_PNR); }

using BKernel = void (*)(BArgs);
static BKernel batched_kernel(int minb) {
    switch (minb) {
        case 4: return slos_batched_kernel<4>;
        case 5: return slos_batched_kernel<5>;
        default: return slos_batched_kernel<6>;
    }
}

struct BatchedPlan {
    int count = 0;
    std::vector<int> m, n, det;
    std::vector<std::vector<int>> s;
    std::vector<int64_t> u_off, out_off;
    std::vector<BShape> shapes;
    std::vector<BLaneGroup> lgs;
    std::string signature;
    // launch configuration (autotuned)
    int chunk = 256, threads = 256, blocks_per_sm = 5, minb = 5;
    // device copies (owned)
    BShape *d_shapes = nullptr;
    BLaneGroup *d_lgs = nullptr;
    BDesc *d_desc = nullptr;
    int64_t *d_first = nullptr, *d_uoff = nullptr, *d_ooff = nullptr;
    uint32_t *d_slots = nullptr;  // transition tables of every shape
    int ndesc = 0;
    int64_t total_items = 0;
    int built_chunk = -1;
    size_t layer_bytes = 0;  // workspace: layer buffers
    size_t ctrl_bytes = 0;   // workspace: counters
    int stall_desc = -1;     // a descriptor that others wait on (fault injection)
    bool inject_stall = false;
};

void batched_destroy(slos_plan_s *p) {
    BatchedPlan *b = p->batched;
    if (!b) return;
    cudaFree(b->d_shapes);
    cudaFree(b->d_lgs);
    cudaFree(b->d_desc);
    cudaFree(b->d_first);
    cudaFree(b->d_uoff);
    cudaFree(b->d_ooff);
    cudaFree(b->d_slots);
    delete b;
    p->batched = nullptr;
}

// Descriptors and item offsets for a given chunk size (host build + upload).
static slos_status_t build_items(BatchedPlan *b, int chunk) {
    if (b->built_chunk == chunk) return SLOS_OK;
    struct D {
        BDesc d;
        int64_t work;
    };
    int kmax = 0;
    for (auto &sh : b->shapes) kmax = std::max(kmax, sh.n);
    std::vector<BDesc> desc;
    std::vector<int> idx_of((size_t)b->lgs.size() * (kmax + 1), -1);
    for (int k = 1; k <= kmax; ++k) {
        std::vector<D> layer;
        for (size_t l = 0; l < b->lgs.size(); ++l) {
            const BShape &sh = b->shapes[b->lgs[l].shape];
            if (k > sh.n) continue;
            D x;
            x.d.lg = (int)l;
            x.d.k = k;
            x.d.dep = -1;
            int64_t nch = 0;
            if (k == sh.n && sh.det == SLOS_DETECT_THRESHOLD) {
                // runs of whole patterns, class by class
                for (int j = 1; j <= sh.nclass; ++j) nch += thresh_items(sh, j, chunk);
            } else {
                // items never straddle a section (slot width)
                for (int sec = 0; sec < kBSec; ++sec)
                    nch += (sh.sec_pos[k][sec + 1] - sh.sec_pos[k][sec] + chunk - 1) / chunk;
            }
            x.d.nchunks = (int)nch;
            x.work = sh.F[k] * std::min(sh.m, k);
            layer.push_back(x);
        }
        std::stable_sort(layer.begin(), layer.end(), [](const D &a, const D &c) { return a.work > c.work; });
        for (auto &x : layer) {
            x.d.dep = k > 1 ? idx_of[(size_t)x.d.lg * (kmax + 1) + k - 1] : -1;
            idx_of[(size_t)x.d.lg * (kmax + 1) + k] = (int)desc.size();
            desc.push_back(x.d);
        }
    }
    std::vector<int64_t> first(desc.size() + 1, 0);
    for (size_t i = 0; i < desc.size(); ++i) first[i + 1] = first[i] + desc[i].nchunks;
    cudaFree(b->d_desc);
    cudaFree(b->d_first);
    b->d_desc = nullptr;
    b->d_first = nullptr;
    if (cudaMalloc(&b->d_desc, std::max<size_t>(1, desc.size()) * sizeof(BDesc)) != cudaSuccess ||
        cudaMalloc(&b->d_first, first.size() * sizeof(int64_t)) != cudaSuccess)
        return fail(SLOS_ERR_OOM, "slos_batched_plan: cannot allocate work descriptors");
    cudaMemcpy(b->d_desc, desc.data(), desc.size() * sizeof(BDesc), cudaMemcpyHostToDevice);
    cudaMemcpy(b->d_first, first.data(), first.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    b->ndesc = (int)desc.size();
    b->total_items = first.back();
    b->stall_desc = -1;
    for (auto &d : desc)
        if (d.dep >= 0) {
            b->stall_desc = d.dep;
            break;
        }
    b->built_chunk = chunk;
    b->ctrl_bytes = align_up(sizeof(unsigned long long)) + align_up((size_t)b->ndesc * sizeof(int));
    return SLOS_OK;
}

static slos_status_t batched_launch(slos_plan_s *p, const void *U, float *out, void *ws, size_t ws_bytes,
                                    cudaStream_t s, int chunk, int threads, int bps, int minb) {
    BatchedPlan *b = p->batched;
    slos_status_t st = build_items(b, chunk);
    if (st != SLOS_OK) return st;
    const size_t need = b->layer_bytes + b->ctrl_bytes;
    if (ws_bytes < need || !ws) return fail(SLOS_ERR_INVALID_ARG, "slos_batched_forward: workspace too small");
    char *w = reinterpret_cast<char *>(ws);
    unsigned long long *head = reinterpret_cast<unsigned long long *>(w + b->layer_bytes);
    int *done = reinterpret_cast<int *>(w + b->layer_bytes + align_up(sizeof(unsigned long long)));
    cudaError_t e;
    if ((e = cudaMemsetAsync(w + b->layer_bytes, 0, b->ctrl_bytes, s)) != cudaSuccess)
        return fail(SLOS_ERR_CUDA, std::string("slos_batched_forward: ") + cudaGetErrorString(e));
    BArgs a;
    a.shapes = b->d_shapes;
    a.lgs = b->d_lgs;
    a.desc = b->d_desc;
    a.first_item = b->d_first;
    a.slots = b->d_slots;
    a.ndesc = b->ndesc;
    a.total_items = b->total_items;
    a.chunk = chunk;
    a.U = reinterpret_cast<const float2 *>(U);
    a.u_off = b->d_uoff;
    a.out = out;
    a.out_off = b->d_ooff;
    a.ws = w;
    a.done = done;
    a.head = head;
    a.status = p->d_status;
    a.spin_limit = 20000000;  // ~4 s of 200 ns sleeps: far beyond any layer
    if (b->inject_stall && b->stall_desc >= 0) {
        // fault injection: this completion counter starts hugely negative, so
        // the items waiting on it never see it complete; short wait limit
        if ((e = cudaMemsetAsync(done + b->stall_desc, 0x80, sizeof(int), s)) != cudaSuccess)
            return fail(SLOS_ERR_CUDA, std::string("slos_batched_forward: ") + cudaGetErrorString(e));
        a.spin_limit = 5000;
    }
    const int warps = threads / 32;
    const size_t smem = (size_t)warps * kBWarpF2 * sizeof(float2);
    const int grid = std::max(1, p->sm_count * bps);
    double bytes = 0.0;
    for (int i = 0; i < b->count; ++i) bytes += 4.0 * (b->out_off[i + 1] - b->out_off[i]);
    ProfScope ps("slos_batched", bytes, s);
    batched_kernel(minb)<<<grid, threads, smem, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return fail(SLOS_ERR_CUDA, std::string("slos_batched_forward: ") + cudaGetErrorString(e));
    return SLOS_OK;
}

// ---------------------------------------------------------------- autotune cache
static std::string device_name(int dev) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    return prop.name;
}

static bool cache_lookup(const std::string &path, const std::string &key, int *chunk, int *threads, int *bps,
                         int *minb) {
    std::ifstream f(path);
    if (!f) return false;
    std::string line;
    while (std::getline(f, line)) {
        // one JSON object per line:
        // {"key": "...", "chunk": C, "threads": T, "blocks_per_sm": B, "min_blocks": R, "ms": X}
        const std::string kq = "\"key\": \"" + key + "\"";
        if (line.find(kq) == std::string::npos) continue;
        auto num = [&](const char *name, int *dst) {
            const std::string nq = std::string("\"") + name + "\": ";
            size_t pos = line.find(nq);
            if (pos == std::string::npos) return false;
            *dst = atoi(line.c_str() + pos + nq.size());
            return true;
        };
        return num("chunk", chunk) && num("threads", threads) && num("blocks_per_sm", bps) && num("min_blocks", minb);
    }
    return false;
}

}  // namespace slos

using namespace slos;

extern "C" {

slos_status_t slos_batched_plan(int count, const int *m, const int *n, const int *const *input_states,
                                const slos_detection_t *detection, slos_plan_t *out) {
    if (!out) return fail(SLOS_ERR_INVALID_ARG, "slos_batched_plan: NULL out");
    *out = nullptr;
    if (count <= 0 || !m || !n || !input_states || !detection)
        return fail(SLOS_ERR_INVALID_ARG, "slos_batched_plan: bad arguments");
    BatchedPlan *b = new BatchedPlan();
    b->count = count;
    std::map<std::vector<int>, int> shape_of;  // (m, det, s...) -> shape index
    std::vector<std::vector<int>> members;
    std::vector<int> shape_idx(count);
    std::ostringstream sig;
    for (int i = 0; i < count; ++i) {
        const int mi = m[i], ni = n[i];
        if (mi < 2 || mi > kBMax || ni < 1 || ni > kMaxPhotons) {
            delete b;
            return fail(SLOS_ERR_UNSUPPORTED, "slos_batched_plan: instance " + std::to_string(i) +
                                                  " needs 2 <= m <= 20 and 1 <= n <= 12");
        }
        if (detection[i] != SLOS_DETECT_PNR && detection[i] != SLOS_DETECT_THRESHOLD) {
            delete b;
            return fail(SLOS_ERR_INVALID_ARG, "slos_batched_plan: unknown detection");
        }
        std::vector<int> key = {mi, (int)detection[i]};
        int tot = 0;
        for (int q = 0; q < mi; ++q) {
            if (input_states[i][q] < 0) {
                delete b;
                return fail(SLOS_ERR_INVALID_ARG, "slos_batched_plan: negative occupation");
            }
            tot += input_states[i][q];
            key.push_back(input_states[i][q]);
        }
        if (tot != ni) {
            delete b;
            return fail(SLOS_ERR_INVALID_ARG, "slos_batched_plan: input state of instance " + std::to_string(i) +
                                                  " does not hold n photons");
        }
        auto it = shape_of.find(key);
        int si;
        if (it == shape_of.end()) {
            si = (int)b->shapes.size();
            shape_of[key] = si;
            BShape sh;
            memset(&sh, 0, sizeof(sh));
            sh.m = mi;
            sh.n = ni;
            sh.det = (int)detection[i];
            int c = 0;
            double sf = 1.0;
            for (int q = 0; q < mi; ++q)
                for (int r = 0; r < input_states[i][q]; ++r) {
                    sh.cols[c++] = q;
                    if (r >= 1) sf *= (r + 1);
                }
            sh.inv_sfact = (float)(1.0 / sf);
            for (int k = 0; k <= ni; ++k) sh.F[k] = binom_host(mi + k - 1, k);
            if (sh.F[ni - 1] >= kBMaxParent) {
                delete b;
                return fail(SLOS_ERR_UNSUPPORTED, "slos_batched_plan: instance " + std::to_string(i) +
                                                      " has more than 2^27 parent states");
            }
            // threshold patterns: classes j = |b| = 1 .. min(n, m), C(m, j) patterns of
            // C(n-1, j-1) final states each (compositions of n into j positive parts)
            int64_t acc = 0, pos = 0;
            sh.nclass = std::min(ni, mi);
            for (int j = 1; j <= sh.nclass; ++j) {
                sh.pat_off[j] = (int)acc;
                sh.pat_cnt[j] = (int)binom_host(ni - 1, j - 1);
                sh.pat_base[j] = pos;
                acc += binom_host(mi, j);
                pos += binom_host(mi, j) * sh.pat_cnt[j];
            }
            sh.pat_off[sh.nclass + 1] = (int)acc;
            sh.K = (int)(detection[i] == SLOS_DETECT_PNR ? sh.F[ni] : acc);
            b->shapes.push_back(sh);
            members.emplace_back();
        } else {
            si = it->second;
        }
        members[si].push_back(i);
        shape_idx[i] = si;
        b->m.push_back(mi);
        b->n.push_back(ni);
        b->det.push_back((int)detection[i]);
        b->s.emplace_back(input_states[i], input_states[i] + mi);
        sig << mi << "," << ni << "," << (int)detection[i] << ";";
    }
    // packed offsets in instance order
    b->u_off.assign(count + 1, 0);
    b->out_off.assign(count + 1, 0);
    for (int i = 0; i < count; ++i) {
        b->u_off[i + 1] = b->u_off[i] + (int64_t)b->m[i] * b->m[i];
        b->out_off[i + 1] = b->out_off[i] + b->shapes[shape_idx[i]].K;
    }
    // lane groups and their layer buffers
    size_t off = 0;
    for (size_t si = 0; si < members.size(); ++si) {
        const BShape &sh = b->shapes[si];
        // groups of 16; the remainder r in 16-wide (r > 12), 8 + 4 (r = 9..12), 8 (r = 5..8) or 4 (r <= 4)
        // groups, so few lanes sit idle (a group's cost is its lanes x its shape's states)
        for (size_t q = 0; q < members[si].size();) {
            BLaneGroup g;
            g.shape = (int)si;
            const size_t r = members[si].size() - q;
            g.width = r > 12 ? kBLanes : (r > 4 ? 8 : 4);
            for (int l = 0; l < kBLanes; ++l)
                g.inst[l] = (l < g.width && q + l < members[si].size()) ? members[si][q + l] : -1;
            q += g.width;
            const int64_t f1 = sh.n >= 2 ? sh.F[sh.n - 1] : 1;
            const int64_t f2 = sh.n >= 3 ? sh.F[sh.n - 2] : 1;
            const size_t b1 = (size_t)f2 * g.width * sizeof(float2);
            g.buf[0] = (int64_t)off;
            off += align_up((size_t)f1 * g.width * sizeof(float2));
            g.buf[1] = (int64_t)off;
            off += align_up(b1);
            b->lgs.push_back(g);
        }
    }
    b->layer_bytes = off;
    // tables: per shape, layers 1..n of slots and the final weights
    int64_t tab_elems = 0;
    int64_t max_sorted = 0;  // largest sorted layer (plan-time scratch)
    for (auto &sh : b->shapes) {
        for (int k = 1; k <= sh.n; ++k) {
            sh.kw[k] = (std::min(sh.m, k) + 1) & ~1;
            sh.slot_off[k] = tab_elems;
            int64_t off = 0;
            if (layer_sorted(sh, k)) {
                // states of layer k with q occupied modes: C(m, q) C(k-1, q-1)
                max_sorted = std::max(max_sorted, sh.F[k]);
                sh.sec_pos[k][0] = 0;
                for (int sec = 0; sec < kBSec; ++sec) {
                    const int q = sec + 1;
                    const int64_t cnt = q <= std::min(sh.m, k) ? binom_host(sh.m, q) * binom_host(k - 1, q - 1) : 0;
                    sh.sec_pos[k][sec + 1] = sh.sec_pos[k][sec] + (int)cnt;
                    off = (off + 3) & ~int64_t(3);  // 16-byte aligned rows for the uint4 reads
                    sh.sec_off[k][sec] = off;
                    off += cnt * sec_width(sec);
                }
            } else {
                const int su = sh.kw[k] - 1;
                for (int sec = 0; sec <= kBSec; ++sec) sh.sec_pos[k][sec] = sec <= su ? 0 : (int)sh.F[k];
                off = sh.F[k] * sh.kw[k];
            }
            tab_elems += (off + 3) & ~int64_t(3);
        }
        if (sh.det == SLOS_DETECT_THRESHOLD && sh.n >= 2)
            for (int j = 1; j <= sh.nclass; ++j)
                if (sh.sec_pos[sh.n][j - 1] != sh.pat_base[j]) {
                    delete b;
                    return fail(SLOS_ERR_INTERNAL, "slos_batched_plan: pattern classes do not match the sections");
                }
        const int64_t fn4 = (sh.F[sh.n] + 3) & ~int64_t(3);
        sh.w_off = tab_elems;
        tab_elems += fn4;
    }
    b->signature = sig.str();
    slos_plan_s *p = new slos_plan_s();
    p->kind = 1;
    p->m = 0;
    p->n = 0;
    p->batched = b;
    p->d_status = nullptr;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete b;
        delete p;
        return fail(SLOS_ERR_CUDA, "slos_batched_plan: no CUDA device");
    }
    cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device);
    if (p->sm_count <= 0) p->sm_count = 148;
    auto cleanup = [&](const char *msg) {
        batched_destroy(p);
        if (p->d_status) cudaFree(p->d_status);
        delete p;
        return fail(SLOS_ERR_OOM, msg);
    };
    if (cudaMalloc(&p->d_status, 64) != cudaSuccess) return cleanup("slos_batched_plan: status word");
    cudaMemset(p->d_status, 0, 64);
    if (cudaMalloc(&b->d_shapes, b->shapes.size() * sizeof(BShape)) != cudaSuccess ||
        cudaMalloc(&b->d_lgs, b->lgs.size() * sizeof(BLaneGroup)) != cudaSuccess ||
        cudaMalloc(&b->d_uoff, b->u_off.size() * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc(&b->d_ooff, b->out_off.size() * sizeof(int64_t)) != cudaSuccess)
        return cleanup("slos_batched_plan: descriptor tables");
    cudaMemcpy(b->d_shapes, b->shapes.data(), b->shapes.size() * sizeof(BShape), cudaMemcpyHostToDevice);
    cudaMemcpy(b->d_lgs, b->lgs.data(), b->lgs.size() * sizeof(BLaneGroup), cudaMemcpyHostToDevice);
    cudaMemcpy(b->d_uoff, b->u_off.data(), b->u_off.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    cudaMemcpy(b->d_ooff, b->out_off.data(), b->out_off.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (cudaMalloc(&b->d_slots, (size_t)tab_elems * sizeof(uint32_t)) != cudaSuccess)
        return cleanup("slos_batched_plan: transition tables");
    // plan-time scratch: positions of two consecutive layers, per-block section counts
    const int64_t max_blk = (max_sorted + 255) / 256;
    int *d_pos[2] = {nullptr, nullptr};
    int *d_cnt = nullptr, *d_base = nullptr;
    auto free_scratch = [&]() {
        cudaFree(d_pos[0]);
        cudaFree(d_pos[1]);
        cudaFree(d_cnt);
        cudaFree(d_base);
    };
    if (max_sorted > 0 &&
        (cudaMalloc(&d_pos[0], (size_t)max_sorted * sizeof(int)) != cudaSuccess ||
         cudaMalloc(&d_pos[1], (size_t)max_sorted * sizeof(int)) != cudaSuccess ||
         cudaMalloc(&d_cnt, (size_t)max_blk * kBSec * sizeof(int)) != cudaSuccess ||
         cudaMalloc(&d_base, (size_t)max_blk * kBSec * sizeof(int)) != cudaSuccess)) {
        free_scratch();
        return cleanup("slos_batched_plan: plan-time scratch");
    }
    std::vector<int> hcnt, hbase;
    for (auto &sh : b->shapes) {
        const int *ppos = nullptr;
        for (int k = 1; k <= sh.n; ++k) {
            const int bs = 256;
            const unsigned grid = (unsigned)((sh.F[k] + bs - 1) / bs);
            int *cpos = nullptr;
            const bool listed = k == sh.n && sh.det == SLOS_DETECT_THRESHOLD;  // list order, no sort pass
            if (layer_sorted(sh, k) && !listed) {
                cpos = d_pos[k & 1];
                section_pass_kernel<kBMax><<<grid, bs>>>(sh, k, d_cnt, nullptr, nullptr);
                hcnt.resize((size_t)grid * kBSec);
                hbase.resize((size_t)grid * kBSec);
                if (cudaMemcpy(hcnt.data(), d_cnt, hcnt.size() * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
                    free_scratch();
                    return cleanup("slos_batched_plan: sorting a layer by occupied modes failed");
                }
                bool ok = true;
                for (int sec = 0; sec < kBSec; ++sec) {
                    int64_t run = sh.sec_pos[k][sec];
                    for (unsigned blk = 0; blk < grid; ++blk) {
                        hbase[(size_t)blk * kBSec + sec] = (int)run;
                        run += hcnt[(size_t)blk * kBSec + sec];
                    }
                    ok = ok && run == sh.sec_pos[k][sec + 1];  // the closed-form section sizes
                }
                if (!ok) {
                    free_scratch();
                    return cleanup("slos_batched_plan: section sizes disagree with C(m, q) C(k-1, q-1)");
                }
                cudaMemcpy(d_base, hbase.data(), hbase.size() * sizeof(int), cudaMemcpyHostToDevice);
                section_pass_kernel<kBMax><<<grid, bs>>>(sh, k, nullptr, d_base, cpos);
            }
            float *w = k == sh.n ? reinterpret_cast<float *>(b->d_slots + sh.w_off) : nullptr;
            build_slots_kernel<kBMax><<<grid, bs>>>(sh, k, b->d_slots + sh.slot_off[k], ppos, cpos, w, listed);
            ppos = cpos;
        }
    }
    const bool built = cudaStreamSynchronize(0) == cudaSuccess && cudaGetLastError() == cudaSuccess;
    free_scratch();
    if (!built) return cleanup("slos_batched_plan: building the transition tables failed");
    slos_status_t st = build_items(b, b->chunk);
    if (st != SLOS_OK) {
        batched_destroy(p);
        cudaFree(p->d_status);
        delete p;
        return st;
    }
    *out = p;
    return SLOS_OK;
}

slos_status_t slos_batched_query(slos_plan_t p, int64_t *u_offsets, int64_t *out_offsets, size_t *workspace_bytes) {
    if (!p || p->kind != 1 || !p->batched) return fail(SLOS_ERR_INVALID_ARG, "slos_batched_query: not a batched plan");
    BatchedPlan *b = p->batched;
    if (u_offsets) memcpy(u_offsets, b->u_off.data(), b->u_off.size() * sizeof(int64_t));
    if (out_offsets) memcpy(out_offsets, b->out_off.data(), b->out_off.size() * sizeof(int64_t));
    if (workspace_bytes) {
        // enough for the largest chunk the autotuner tries (smallest chunk = most descriptors is the same count)
        *workspace_bytes = b->layer_bytes + align_up(sizeof(unsigned long long)) +
                           align_up((size_t)b->lgs.size() * (kMaxPhotons + 1) * sizeof(int));
    }
    return SLOS_OK;
}

slos_status_t slos_batched_forward(slos_plan_t p, const void *U_packed, float *out_packed, void *workspace,
                                   size_t workspace_bytes, void *stream) {
    if (!p || p->kind != 1 || !p->batched) return fail(SLOS_ERR_INVALID_ARG, "slos_batched_forward: not a batched plan");
    if (!U_packed || !out_packed) return fail(SLOS_ERR_INVALID_ARG, "slos_batched_forward: NULL pointer");
    BatchedPlan *b = p->batched;
    return batched_launch(p, U_packed, out_packed, workspace, workspace_bytes, (cudaStream_t)stream, b->chunk,
                          b->threads, b->blocks_per_sm, b->minb);
}

slos_status_t slos_batched_inject_stall(slos_plan_t p, int enable) {
    if (!p || p->kind != 1 || !p->batched) return fail(SLOS_ERR_INVALID_ARG, "slos_batched_inject_stall: not a batched plan");
    p->batched->inject_stall = enable != 0;
    return SLOS_OK;
}

slos_status_t slos_batched_autotune(slos_plan_t p, const void *U_packed, float *out_packed, void *workspace,
                                    size_t workspace_bytes, const char *cache_path, void *stream) {
    if (!p || p->kind != 1 || !p->batched) return fail(SLOS_ERR_INVALID_ARG, "slos_batched_autotune: not a batched plan");
    BatchedPlan *b = p->batched;
    cudaStream_t s = (cudaStream_t)stream;
    const std::string key = device_name(p->device) + "|" + std::to_string(std::hash<std::string>()(b->signature));
    int c = 0, t = 0, bp = 0, mb = 0;
    if (cache_path && cache_lookup(cache_path, key, &c, &t, &bp, &mb)) {
        b->chunk = c;
        b->threads = t;
        b->blocks_per_sm = bp;
        b->minb = mb;
        return build_items(b, c);
    }
    const int chunks[] = {128, 256, 512};
    const int thread_opts[] = {128, 256};
    const int minb_opts[] = {4, 5, 6};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int bc = b->chunk, bt = b->threads, bb = b->blocks_per_sm, bm = b->minb;
    for (int mbv : minb_opts) {
        for (int th : thread_opts) {
            int nb = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batched_kernel(mbv), th,
                                                          (size_t)(th / 32) * kBWarpF2 * sizeof(float2));
            // a persistent grid must be fully resident: all of it, or one block per SM less
            for (int bps = std::max(1, nb - 1); bps <= nb; ++bps) {
                for (int ch : chunks) {
                    slos_status_t st =
                        batched_launch(p, U_packed, out_packed, workspace, workspace_bytes, s, ch, th, bps, mbv);
                    if (st != SLOS_OK) return st;  // warm-up (also builds the items)
                    cudaEventRecord(e0, s);
                    for (int r = 0; r < 2; ++r) {
                        st = batched_launch(p, U_packed, out_packed, workspace, workspace_bytes, s, ch, th, bps, mbv);
                        if (st != SLOS_OK) return st;
                    }
                    cudaEventRecord(e1, s);
                    if (cudaEventSynchronize(e1) != cudaSuccess) return fail(SLOS_ERR_CUDA, "slos_batched_autotune: sync");
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    ms *= 0.5f;
                    if (ms < best) {
                        best = ms;
                        bc = ch;
                        bt = th;
                        bb = bps;
                        bm = mbv;
                    }
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->chunk = bc;
    b->threads = bt;
    b->blocks_per_sm = bb;
    b->minb = bm;
    if (cache_path) {
        std::ofstream f(cache_path, std::ios::app);
        if (f) {
            f << "{\"key\": \"" << key << "\", \"chunk\": " << bc << ", \"threads\": " << bt
              << ", \"blocks_per_sm\": " << bb << ", \"min_blocks\": " << bm << ", \"ms\": " << best << "}\n";
        }
    }
    return build_items(b, bc);
}

}  // extern "C"
