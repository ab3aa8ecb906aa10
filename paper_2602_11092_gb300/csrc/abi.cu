// C-ABI entry points: plans, forward/backward orchestration, mesh calls and
// the exact index tables.  Every stream operation is asynchronous; nothing
// here allocates on the forward/backward path.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <fstream>
#include <mutex>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/slos.h"
#include "common.cuh"
#include "mesh.h"
#include "plan.h"
#include "profile.h"
#include "slos_kernels.cuh"
#include "fused.h"
#include "prefix.h"
#include "split.h"
#include "tab_launch.h"

namespace slos {

SLOS_DECLARE_LAUNCHERS(8)
SLOS_DECLARE_LAUNCHERS(12)
SLOS_DECLARE_LAUNCHERS(16)
SLOS_DECLARE_LAUNCHERS(20)
SLOS_DECLARE_LAUNCHERS(24)

static thread_local std::string g_last_error;

slos_status_t fail(slos_status_t st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

#define SLOS_CUDA(call)                                                                             \
    do {                                                                                            \
        cudaError_t e__ = (call);                                                                   \
        if (e__ != cudaSuccess)                                                                     \
            return fail(SLOS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e__));     \
    } while (0)

// Plan-time host-to-device copy; false on failure.
static bool h2d(void *dst, const void *src, size_t bytes) {
    return cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
}

static int mmax_for(int m) {
    if (m <= 8) return 8;
    if (m <= 12) return 12;
    if (m <= 16) return 16;
    if (m <= 20) return 20;
    return 24;
}

cudaError_t launch_fwd(int m, const FwdArgs &a, int epi, bool save, int bx, cudaStream_t s) {
    switch (mmax_for(m)) {
        case 8: return slos_launch_fwd_m8(a, epi, save, bx, s);
        case 12: return slos_launch_fwd_m12(a, epi, save, bx, s);
        case 16: return slos_launch_fwd_m16(a, epi, save, bx, s);
        case 20: return slos_launch_fwd_m20(a, epi, save, bx, s);
        default: return slos_launch_fwd_m24(a, epi, save, bx, s);
    }
}
cudaError_t launch_bwd(int m, const BwdArgs &a, int seed, int bx, cudaStream_t s) {
    switch (mmax_for(m)) {
        case 8: return slos_launch_bwd_m8(a, seed, bx, s);
        case 12: return slos_launch_bwd_m12(a, seed, bx, s);
        case 16: return slos_launch_bwd_m16(a, seed, bx, s);
        case 20: return slos_launch_bwd_m20(a, seed, bx, s);
        default: return slos_launch_bwd_m24(a, seed, bx, s);
    }
}
cudaError_t launch_prep(int m, const PrepArgs &a, int bx, bool bcast, cudaStream_t s) {
    switch (mmax_for(m)) {
        case 8: return slos_launch_prep_m8(a, bx, bcast, s);
        case 12: return slos_launch_prep_m12(a, bx, bcast, s);
        case 16: return slos_launch_prep_m16(a, bx, bcast, s);
        case 20: return slos_launch_prep_m20(a, bx, bcast, s);
        default: return slos_launch_prep_m24(a, bx, bcast, s);
    }
}
cudaError_t launch_bwd_tab(int m, const BwdArgs &a, const int32_t *ctab, int seed, int bx, bool holes, cudaStream_t s) {
    switch (mmax_for(m)) {
        case 8: return slos_launch_bwd_tab_m8(a, ctab, seed, bx, holes, s);
        case 12: return slos_launch_bwd_tab_m12(a, ctab, seed, bx, holes, s);
        case 16: return slos_launch_bwd_tab_m16(a, ctab, seed, bx, holes, s);
        case 20: return slos_launch_bwd_tab_m20(a, ctab, seed, bx, holes, s);
        default: return slos_launch_bwd_tab_m24(a, ctab, seed, bx, holes, s);
    }
}

static cudaError_t init_device_once(int dev) {
    static std::mutex mu;
    static bool done[64] = {false};
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return cudaSuccess;
    cudaError_t e;
    if ((e = slos_init_m8()) != cudaSuccess) return e;
    if ((e = slos_init_m12()) != cudaSuccess) return e;
    if ((e = slos_init_m16()) != cudaSuccess) return e;
    if ((e = slos_init_m20()) != cudaSuccess) return e;
    if ((e = slos_init_m24()) != cudaSuccess) return e;
    if ((e = slos_fused_init()) != cudaSuccess) return e;
    if ((e = slos_pair_init()) != cudaSuccess) return e;
    if ((e = slos_prefix_init()) != cudaSuccess) return e;
    done[dev] = true;
    return cudaSuccess;
}

// ------------------------------------------------------------------ host fault injection
// Test hooks (slos_inject_fault): they make host calls fail as the real
// failure would, so error paths are exercised without faulting a GPU.
static std::atomic<int> g_inject_alloc{0};         // n > 0: the n-th plan-time allocation from now fails
static std::atomic<int> g_inject_stream_dev{-1};   // >= 0: stream device queries report this device
static std::atomic<int> g_inject_table_budget{0};  // 1: every plan finds its table budget exceeded

// Device allocation made while building a plan.
static cudaError_t plan_malloc(void **ptr, size_t bytes) {
    if (g_inject_alloc.load() > 0 && g_inject_alloc.fetch_sub(1) == 1) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(ptr, bytes);
}
template <typename T>
static cudaError_t plan_malloc(T **ptr, size_t bytes) {
    return plan_malloc(reinterpret_cast<void **>(ptr), bytes);
}

// The stream must belong to the plan's device (its tables live there).  A
// stream that is being captured into a graph is not asked (a device query
// there ends the capture with an error), and a query that cannot answer is
// not treated as a mismatch.
static slos_status_t check_stream(const slos_plan_s *p, cudaStream_t s, const char *who) {
    int dev = g_inject_stream_dev.load();
    if (dev < 0) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
            cudaGetLastError();
            return SLOS_OK;
        }
        if (cs != cudaStreamCaptureStatusNone) return SLOS_OK;
        if (cudaStreamGetDevice(s, &dev) != cudaSuccess) {
            cudaGetLastError();
            return SLOS_OK;
        }
    }
    if (dev != p->device)
        return fail(SLOS_ERR_INVALID_ARG, std::string(who) + ": the stream belongs to device " + std::to_string(dev) +
                                              " but the plan was built on device " + std::to_string(p->device));
    return SLOS_OK;
}

// Every index of a layer's slot table and child table in range before upload:
// a slot names a parent of layer k-1 and a mode, or is padding; every state
// has at least one parent; a child entry names a state of layer k (or -1
// where the lattice has no such child, if holes are allowed).
static bool tables_in_range(int m, int64_t Fprev, int64_t Fk, int kw, const uint32_t *slots, const int32_t *ctab,
                            bool holes, std::string *why) {
    for (int64_t c = 0; c < Fk; ++c) {
        int occ = 0;
        for (int q = 0; q < kw; ++q) {
            const uint32_t e = slots[(size_t)c * kw + q];
            if (e == kSlotEmpty) continue;
            if ((int)(e & 31u) >= m || (int64_t)(e >> 5) >= Fprev) {
                *why = "slot " + std::to_string(q) + " of state " + std::to_string(c) + " out of range";
                return false;
            }
            ++occ;
        }
        if (occ == 0) {
            *why = "state " + std::to_string(c) + " has no parent";
            return false;
        }
    }
    for (int64_t i = 0; i < Fprev * m; ++i) {
        const int32_t x = ctab[i];
        if (x >= Fk || x < (holes ? -1 : 0)) {
            *why = "child entry " + std::to_string(i) + " out of range";
            return false;
        }
    }
    return true;
}

// ------------------------------------------------------------------ host index
int64_t binom_host(int a, int e) {
    if (e < 0 || a < 0 || e > a) return 0;
    int64_t r = 1;
    for (int i = 1; i <= e; ++i) r = r * (a - e + i) / i;
    return r;
}

// rank(t) = sum_b C(p_b, m-1-b), p_b = distance of bar b from the string end.
int64_t host_rank(int m, const int *t) {
    int64_t r = 0;
    int after = 0;  // stars after bar b
    // p_b = (stars after bar b) + (bars after bar b) = R_b + (m-2-b)
    for (int b = m - 2; b >= 0; --b) {
        after += t[b + 1];
        r += binom_host(after + (m - 2 - b), m - 1 - b);
    }
    return r;
}

void host_unrank(int m, int k, int64_t r, int *t) {
    const int L = k + m - 1;
    std::vector<int> p(m + 1);
    int x = L - 1;
    for (int b = 0; b < m - 1; ++b) {
        const int e = m - 1 - b;
        while (binom_host(x, e) > r) --x;
        p[b] = x;
        r -= binom_host(x, e);
        --x;
    }
    for (int j = 0; j < m; ++j) {
        const int hi = (j == 0) ? L : p[j - 1];
        const int lo = (j < m - 1) ? p[j] : -1;
        t[j] = hi - lo - 1;
    }
}


// ------------------------------------------------------------------ transition graph
// Built on the host by walking each layer in descending-lex order with the
// bar mask (next larger integer with the same popcount) and the closed-form
// parent/child rank offsets, then uploaded once.
static uint64_t next_comb_host(uint64_t z) {
    const uint64_t c = z & (0ull - z);
    const uint64_t r = z + c;
    return r | (((r ^ z) >> 2) >> __builtin_ctzll(z));
}

static void bars_of(uint64_t z, int m, int L, int *p, int *t) {
    // p[b]: b-th highest set bit; t[j] = p[j-1] - p[j] - 1
    int b = 0;
    for (int q = L - 1; q >= 0 && b < m - 1; --q)
        if ((z >> q) & 1ull) p[b++] = q;
    for (int j = 0; j < m; ++j) {
        const int hi = (j == 0) ? L : p[j - 1];
        const int lo = (j < m - 1) ? p[j] : -1;
        t[j] = hi - lo - 1;
    }
}

static void free_fused_tables(slos_plan_s *p) {
    for (auto &L : p->tab.fused) {
        if (L.rows) cudaFree(L.rows);
        if (L.blk) cudaFree(L.blk);
    }
    p->tab.fused.clear();
    if (p->tab.fused_id) cudaFree(p->tab.fused_id);
    if (p->tab.fused_w) cudaFree(p->tab.fused_w);
    p->tab.fused_id = nullptr;
    p->tab.fused_w = nullptr;
}

static void free_split_tables(slos_plan_s *p) {
    SplitTables *st = p->split;
    if (!st) return;
    for (auto &L : st->layer) {
        cudaFree(L.bdesc);
        cudaFree(L.bhead);
        cudaFree(L.bchunk);
    }
    cudaFree(st->tctab);
    delete st;
    p->split = nullptr;
}

static void free_tables(slos_plan_s *p) {
    free_split_tables(p);
    free_fused_tables(p);
    for (auto &L : p->tab.layer) {
        if (L.slots) cudaFree(L.slots);
        if (L.ctab) cudaFree(L.ctab);
        if (L.colinfo) cudaFree(L.colinfo);
        L = LayerTables();
    }
    if (p->tab.w) cudaFree(p->tab.w);
    if (p->tab.occ) cudaFree(p->tab.occ);
    if (p->tab.gfact) cudaFree(p->tab.gfact);
    cudaFree(p->tab.lrank);
    cudaFree(p->tab.lpat);
    cudaFree(p->tab.lw);
    cudaFree(p->tab.lseg);
    p->tab.lrank = p->tab.lpat = p->tab.lseg = nullptr;
    p->tab.lw = nullptr;
    p->tab.nseg = 0;
    p->tab.gfact = nullptr;
    p->tab.w = nullptr;
    p->tab.occ = nullptr;
    p->tab.enabled = false;
}

// Threshold detection: list position of every final state (n photons, m
// modes) in the pattern-grouped order of tables.h.  A state with support b
// (j = |b| modes) sits at
//     base_j + colex(b) C(n-1, j-1) + rank(u),  u = t - 1_b on the modes of b,
// where base_j counts the states of the patterns with fewer modes and rank(u)
// is u's descending-lex rank among the compositions of n - j over j modes.
// Also the work items of the final layer: runs of whole patterns of about
// kThreshSegStates states (at least one pattern), so that one warp sums each
// pattern.
constexpr int kThreshSegStates = 48;
static void threshold_list_host(int m, int n, std::vector<int32_t> &pos, std::vector<int32_t> &seg) {
    const int64_t Fn = binom_host(m + n - 1, n);
    const int jmax = std::min(m, n);
    std::vector<int64_t> base(jmax + 2, 0);
    for (int j = 1; j <= jmax; ++j) base[j + 1] = base[j] + binom_host(m, j) * binom_host(n - 1, j - 1);
    pos.assign(Fn, 0);
    std::vector<int> bar(m + 1), t(m + 1), u(m + 1);
    uint64_t z = 0;
    for (int b = 0; b < m - 1; ++b) z |= 1ull << b;
    for (int64_t c = 0; c < Fn; ++c) {
        bars_of(z, m, n + m - 1, bar.data(), t.data());
        int j = 0;
        int64_t colex = 0;
        for (int q = 0; q < m; ++q)
            if (t[q] > 0) {
                u[j] = t[q] - 1;
                ++j;
                colex += binom_host(q, j);
            }
        pos[c] = (int32_t)(base[j] + colex * binom_host(n - 1, j - 1) + host_rank(j, u.data()));
        z = next_comb_host(z);
    }
    seg.clear();
    for (int j = 1; j <= jmax; ++j) {
        const int64_t cnt = binom_host(n - 1, j - 1), npat = binom_host(m, j);
        const int64_t per = std::max<int64_t>(1, kThreshSegStates / cnt);
        for (int64_t q = 0; q < npat; q += per) seg.push_back((int32_t)(base[j] + q * cnt));
    }
    seg.push_back((int32_t)Fn);
}

// Transition graph of layer k (k photons, m modes) on the host: CSR parent
// entries of every child state and the child table of every parent state.
static void build_layer_host(int m, int k, std::vector<int32_t> &rowptr, std::vector<uint32_t> &entries,
                             std::vector<int32_t> &ctab) {
    const int64_t Fk = binom_host(m + k - 1, k), Fp = binom_host(m + k - 2, k - 1);
    std::vector<int> bar(m + 1), t(m + 1);
    uint64_t first = 0;  // (k, 0, ..., 0): all bars packed at the end of the string
    for (int b = 0; b < m - 1; ++b) first |= 1ull << b;
    const int L = k + m - 1;
    rowptr.assign(Fk + 1, 0);
    entries.clear();
    entries.reserve((size_t)m * Fp);
    uint64_t z = first;
    for (int64_t c = 0; c < Fk; ++c) {
        bars_of(z, m, L, bar.data(), t.data());
        rowptr[c] = (int32_t)entries.size();
        int64_t S = 0;
        for (int j = 0; j < m; ++j) {
            if (t[j] > 0) entries.push_back((uint32_t)((c - S) << 6) | (uint32_t)(j << 1));
            if (j < m - 1) S += bar[j] > 0 ? binom_host(bar[j] - 1, m - 2 - j) : 0;
        }
        entries.back() |= 1u;
        z = next_comb_host(z);
    }
    rowptr[Fk] = (int32_t)entries.size();
    const int Lp = (k - 1) + m - 1;
    ctab.assign((size_t)Fp * m, 0);
    if (k == 1) {
        for (int j = 0; j < m; ++j) ctab[j] = j;  // vacuum -> e_j has rank j
        return;
    }
    z = first;
    for (int64_t c = 0; c < Fp; ++c) {
        bars_of(z, m, Lp, bar.data(), t.data());
        int64_t S = 0;
        for (int j = 0; j < m; ++j) {
            ctab[(size_t)c * m + j] = (int32_t)(c + S);
            if (j < m - 1) S += binom_host(bar[j], m - 2 - j);
        }
        z = next_comb_host(z);
    }
}

// Collision-free lattice (slos_space_t UNBUNCHED): the states of k photons
// are the k-subsets S of the modes, listed in descending lexicographic order
// of their occupation vectors (= ascending lexicographic order of the sorted
// subsets); position of t = sum over empty modes i with r_i > 0 occupied modes
// at or after i of C(m - i - 1, r_i - 1).  Every parent S \ {j} is in the
// lattice; a child S + {j} is not when j is in S (child table entry -1).
static int64_t unbunched_rank(const std::vector<int> &t, int m) {
    int64_t r = 0;
    int after = 0;
    std::vector<int> ones_after(m + 1, 0);
    for (int i = m - 1; i >= 0; --i) ones_after[i] = ones_after[i + 1] + t[i];
    for (int i = 0; i < m; ++i) {
        after = ones_after[i];
        if (t[i] == 0 && after >= 1) r += binom_host(m - i - 1, after - 1);
    }
    return r;
}

// next k-subset in ascending lexicographic order; false after the last
static bool next_subset(std::vector<int> &S, int m) {
    const int k = (int)S.size();
    int i = k - 1;
    while (i >= 0 && S[i] == m - k + i) --i;
    if (i < 0) return false;
    ++S[i];
    for (int q = i + 1; q < k; ++q) S[q] = S[q - 1] + 1;
    return true;
}

static slos_status_t build_tables_unbunched(slos_plan_s *p) {
    const int m = p->m, n = p->n;
    size_t bytes = 0;
    for (int k = 1; k <= n; ++k) bytes += 4 * (size_t)p->F[k] * slot_width(m, k) + 4 * (size_t)m * p->F[k - 1];
    bytes += 4 * (size_t)p->F[n] + (size_t)p->K * m;
    if (bytes > kTableBudgetBytes || p->F[n] >= ((int64_t)1 << 26))
        return fail(SLOS_ERR_UNSUPPORTED, "slos_plan_space: collision-free space too large for transition tables");
    p->tab.layer.assign(n + 1, LayerTables());
    std::vector<int> t(m);
    for (int k = 1; k <= n; ++k) {
        const int kw = slot_width(m, k);
        std::vector<uint32_t> slots((size_t)p->F[k] * kw, kSlotEmpty);
        std::vector<int32_t> ctab((size_t)p->F[k - 1] * m, -1);
        // parents' child rows: every (k-1)-subset in order, every mode
        {
            std::vector<int> S(k - 1);
            for (int q = 0; q < k - 1; ++q) S[q] = q;
            int64_t c = 0;
            do {
                std::fill(t.begin(), t.end(), 0);
                for (int q : S) t[q] = 1;
                for (int j = 0; j < m; ++j) {
                    if (t[j]) continue;
                    t[j] = 1;
                    ctab[(size_t)c * m + j] = (int32_t)unbunched_rank(t, m);
                    t[j] = 0;
                }
                ++c;
            } while (k - 1 > 0 && next_subset(S, m));
        }
        // states' parent slots
        {
            std::vector<int> S(k);
            for (int q = 0; q < k; ++q) S[q] = q;
            int64_t c = 0;
            do {
                std::fill(t.begin(), t.end(), 0);
                for (int q : S) t[q] = 1;
                int q = 0;
                for (int j : S) {
                    t[j] = 0;
                    slots[(size_t)c * kw + q++] = ((uint32_t)unbunched_rank(t, m) << 5) | (uint32_t)j;
                    t[j] = 1;
                }
                ++c;
            } while (next_subset(S, m));
        }
        LayerTables &LT = p->tab.layer[k];
        LT.kw = kw;
        {
            std::string why;
            if (!tables_in_range(m, p->F[k - 1], p->F[k], kw, slots.data(), ctab.data(), true, &why)) {
                free_tables(p);
                return fail(SLOS_ERR_INTERNAL, "slos_plan_space: layer " + std::to_string(k) + ": " + why);
            }
        }
        if (plan_malloc(&LT.slots, slots.size() * 4) != cudaSuccess ||
            plan_malloc(&LT.ctab, ctab.size() * 4) != cudaSuccess) {
            free_tables(p);
            return fail(SLOS_ERR_OOM, "slos_plan_space: cannot allocate the transition tables");
        }
        if (!h2d(LT.slots, slots.data(), slots.size() * 4) || !h2d(LT.ctab, ctab.data(), ctab.size() * 4)) {
            free_tables(p);
            return fail(SLOS_ERR_CUDA, "slos_plan_space: cannot upload the transition tables");
        }
    }
    // final layer: prod t! = 1, so every weight is 1 / prod s!
    std::vector<float> w(p->F[n], p->inv_sfact);
    std::vector<uint8_t> occ((size_t)p->K * m, 0);
    {
        std::vector<int> S(n);
        for (int q = 0; q < n; ++q) S[q] = q;
        int64_t c = 0;
        do {
            for (int q : S) occ[(size_t)c * m + q] = 1;
            ++c;
        } while (next_subset(S, m));
    }
    if (plan_malloc(&p->tab.w, w.size() * 4) != cudaSuccess || plan_malloc(&p->tab.occ, occ.size()) != cudaSuccess) {
        free_tables(p);
        return fail(SLOS_ERR_OOM, "slos_plan_space: cannot allocate the weight tables");
    }
    if (!h2d(p->tab.w, w.data(), w.size() * 4) || !h2d(p->tab.occ, occ.data(), occ.size())) {
        free_tables(p);
        return fail(SLOS_ERR_CUDA, "slos_plan_space: cannot upload the weight tables");
    }
    p->tab.bytes = bytes;
    p->tab.enabled = true;
    return SLOS_OK;
}

static slos_status_t build_tables(slos_plan_s *p) {
    if (p->space == SLOS_SPACE_UNBUNCHED) return build_tables_unbunched(p);
    const int m = p->m, n = p->n;
    size_t bytes = 0;
    for (int k = 1; k <= n; ++k) {
        // packed parent ranks < 2^26; 32-bit element offsets (state * 32) in the kernels
        if (p->F[k - 1] >= kMaxTableParent || p->F[k] >= ((int64_t)1 << 27) || p->F[k] >= ((int64_t)1 << 31) / m)
            return SLOS_OK;  // too large: arithmetic-index kernels
        bytes += 4 * (size_t)p->F[k] * slot_width(m, k) + 4 * (size_t)m * p->F[k - 1];
    }
    bytes += 8 * (size_t)p->F[n] + (size_t)p->K * m;
    if (p->det == SLOS_DETECT_THRESHOLD) bytes += 12 * (size_t)p->F[n];  // list-order tables
    if (bytes > kTableBudgetBytes || g_inject_table_budget.load()) return SLOS_OK;  // arithmetic-index kernels
    p->tab.layer.assign(n + 1, LayerTables());
    std::vector<int> bar(m + 1), t(m + 1);
    const bool thresh = p->det == SLOS_DETECT_THRESHOLD;
    std::vector<int32_t> lpos, lseg;
    if (thresh) threshold_list_host(m, n, lpos, lseg);
    auto init_mask = [&](int k) {
        // first state (k, 0, ..., 0): all bars at the end of the string
        uint64_t z = 0;
        for (int b = 0; b < m - 1; ++b) z |= 1ull << b;
        (void)k;
        return z;
    };
    for (int k = 1; k <= n; ++k) {
        std::vector<int32_t> rowptr, ctab;
        std::vector<uint32_t> entries;
        build_layer_host(m, k, rowptr, entries, ctab);
        LayerTables &LT = p->tab.layer[k];
        // CSR -> fixed-width slots (parent << 5 | mode), padded with empty slots
        const int kw = slot_width(m, k);
        std::vector<uint32_t> slots((size_t)p->F[k] * kw, kSlotEmpty);
        for (int64_t c = 0; c < p->F[k]; ++c)
            for (int32_t q = rowptr[c]; q < rowptr[c + 1]; ++q)
                slots[(size_t)c * kw + (q - rowptr[c])] = ((entries[q] >> 6) << 5) | ((entries[q] >> 1) & 31u);
        LT.kw = kw;
        {
            std::string why;
            if (!tables_in_range(m, p->F[k - 1], p->F[k], kw, slots.data(), ctab.data(), false, &why)) {
                free_tables(p);
                return fail(SLOS_ERR_INTERNAL, "slos_plan: layer " + std::to_string(k) + ": " + why);
            }
        }
        if (thresh && k == n) {
            // the final layer's rows in list order
            std::vector<uint32_t> rows(slots.size());
            for (int64_t c = 0; c < p->F[n]; ++c)
                memcpy(&rows[(size_t)lpos[c] * kw], &slots[(size_t)c * kw], kw * sizeof(uint32_t));
            slots.swap(rows);
        }
        if (plan_malloc(&LT.slots, slots.size() * 4) != cudaSuccess ||
            plan_malloc(&LT.ctab, ctab.size() * 4) != cudaSuccess) {
            free_tables(p);
            return fail(SLOS_ERR_OOM, "slos_plan: cannot allocate the transition tables");
        }
        if (!h2d(LT.slots, slots.data(), slots.size() * 4) || !h2d(LT.ctab, ctab.data(), ctab.size() * 4)) {
            free_tables(p);
            return fail(SLOS_ERR_CUDA, "slos_plan: cannot upload the transition tables");
        }
    }
    // final-layer weights and threshold patterns
    {
        const int L = n + m - 1;
        std::vector<float> w(p->F[n]);
        std::vector<int32_t> pat(p->F[n]);
        std::vector<uint8_t> occ((size_t)p->K * m, 0);
        uint64_t z = init_mask(n);
        for (int64_t c = 0; c < p->F[n]; ++c) {
            bars_of(z, m, L, bar.data(), t.data());
            if (p->det == SLOS_DETECT_PNR)
                for (int j = 0; j < m; ++j) occ[(size_t)c * m + j] = (uint8_t)t[j];
            double f = 1.0;
            uint32_t supp = 0;
            for (int j = 0; j < m; ++j) {
                for (int q = 2; q <= t[j]; ++q) f *= q;
                if (t[j] > 0) supp |= 1u << j;
            }
            w[c] = (float)(f * (double)p->inv_sfact);
            int64_t r = 0;
            int i = 1;
            for (int q = 0; q < m; ++q)
                if ((supp >> q) & 1u) r += binom_host(q, i++);
            pat[c] = p->pat_off[__builtin_popcount(supp)] + (int32_t)r;
            if (p->det == SLOS_DETECT_THRESHOLD)
                for (int j = 0; j < m; ++j) occ[(size_t)pat[c] * m + j] = (uint8_t)((supp >> j) & 1u);
            z = next_comb_host(z);
        }
        if (plan_malloc(&p->tab.occ, occ.size()) != cudaSuccess) {
            free_tables(p);
            return fail(SLOS_ERR_OOM, "slos_plan: cannot allocate the occupation table");
        }
        if (!h2d(p->tab.occ, occ.data(), occ.size())) {
            free_tables(p);
            return fail(SLOS_ERR_CUDA, "slos_plan: cannot upload the occupation table");
        }
        if (plan_malloc(&p->tab.w, w.size() * 4) != cudaSuccess) {
            free_tables(p);
            return fail(SLOS_ERR_OOM, "slos_plan: cannot allocate the weight table");
        }
        if (!h2d(p->tab.w, w.data(), w.size() * 4)) {
            free_tables(p);
            return fail(SLOS_ERR_CUDA, "slos_plan: cannot upload the weight table");
        }
        if (thresh) {
            std::vector<int32_t> lrank(p->F[n]), lpat(p->F[n]);
            std::vector<float> lw(p->F[n]);
            for (int64_t c = 0; c < p->F[n]; ++c) {
                lrank[lpos[c]] = (int32_t)c;
                lpat[lpos[c]] = pat[c];
                lw[lpos[c]] = w[c];
            }
            // every pattern lies inside one work item
            for (size_t i = 0; i + 1 < lseg.size(); ++i)
                if (lseg[i] >= lseg[i + 1] || (lseg[i] > 0 && lpat[lseg[i]] == lpat[lseg[i] - 1])) {
                    free_tables(p);
                    return fail(SLOS_ERR_INTERNAL, "slos_plan: threshold work items split a pattern");
                }
            p->tab.nseg = (int)lseg.size() - 1;
            if (plan_malloc(&p->tab.lrank, lrank.size() * 4) != cudaSuccess ||
                plan_malloc(&p->tab.lpat, lpat.size() * 4) != cudaSuccess ||
                plan_malloc(&p->tab.lw, lw.size() * 4) != cudaSuccess ||
                plan_malloc(&p->tab.lseg, lseg.size() * 4) != cudaSuccess) {
                free_tables(p);
                return fail(SLOS_ERR_OOM, "slos_plan: cannot allocate the threshold list tables");
            }
            if (!h2d(p->tab.lrank, lrank.data(), lrank.size() * 4) || !h2d(p->tab.lpat, lpat.data(), lpat.size() * 4) ||
                !h2d(p->tab.lw, lw.data(), lw.size() * 4) || !h2d(p->tab.lseg, lseg.data(), lseg.size() * 4)) {
                free_tables(p);
                return fail(SLOS_ERR_CUDA, "slos_plan: cannot upload the threshold list tables");
            }
        }
    }
    p->tab.bytes = bytes;
    p->tab.enabled = true;
    return SLOS_OK;
}

// Amplitude encoding (slos_encoded_forward): for every state s of every
// layer k, its highest occupied mode c and the rank of s - e_c in layer k-1
// (the column recursion of the transfer matrix), and sqrt(prod t!) of the
// final states.  Built for PNR table plans of at most kMaxEncodeStates
// outputs; an allocation or upload failure fails the plan.
static slos_status_t build_encode_tables(slos_plan_s *p) {
    if (!p->tab.enabled || p->det != SLOS_DETECT_PNR || p->K > kMaxEncodeStates) return SLOS_OK;
    const int m = p->m, n = p->n;
    const bool unb = p->space == SLOS_SPACE_UNBUNCHED;
    std::vector<float> g(p->F[n], 1.f);
    for (int k = 1; k <= n; ++k) {
        std::vector<uint32_t> info(p->F[k]);
        std::vector<int> t(m + 1), bar(m + 1);
        auto emit = [&](int64_t c) {
            int hi = m - 1;
            while (t[hi] == 0) --hi;
            t[hi] -= 1;
            const int64_t r = unb ? unbunched_rank(std::vector<int>(t.begin(), t.begin() + m), m) : host_rank(m, t.data());
            t[hi] += 1;
            info[c] = ((uint32_t)r << 5) | (uint32_t)hi;
            if (k == n) {
                double f = 1.0;
                for (int j = 0; j < m; ++j)
                    for (int q = 2; q <= t[j]; ++q) f *= q;
                g[c] = (float)std::sqrt(f);
            }
        };
        if (unb) {
            std::vector<int> S(k);
            for (int q = 0; q < k; ++q) S[q] = q;
            int64_t c = 0;
            do {
                std::fill(t.begin(), t.end(), 0);
                for (int q : S) t[q] = 1;
                emit(c++);
            } while (next_subset(S, m));
        } else {
            uint64_t z = 0;
            for (int b = 0; b < m - 1; ++b) z |= 1ull << b;
            for (int64_t c = 0; c < p->F[k]; ++c) {
                bars_of(z, m, k + m - 1, bar.data(), t.data());
                emit(c);
                z = next_comb_host(z);
            }
        }
        uint32_t *d = nullptr;
        if (plan_malloc(&d, info.size() * 4) != cudaSuccess)
            return fail(SLOS_ERR_OOM, "slos_plan: cannot allocate the amplitude-encoding tables");
        p->tab.layer[k].colinfo = d;  // owned by the plan from here on (freed with its tables)
        if (!h2d(d, info.data(), info.size() * 4))
            return fail(SLOS_ERR_CUDA, "slos_plan: cannot upload the amplitude-encoding tables");
    }
    if (plan_malloc(&p->tab.gfact, g.size() * 4) != cudaSuccess) {
        p->tab.gfact = nullptr;
        return fail(SLOS_ERR_OOM, "slos_plan: cannot allocate the amplitude-encoding weights");
    }
    if (!h2d(p->tab.gfact, g.data(), g.size() * 4))
        return fail(SLOS_ERR_CUDA, "slos_plan: cannot upload the amplitude-encoding weights");
    return SLOS_OK;
}

// Split-lattice tables (split.h) for Fock table plans of 8..16 modes: head
// block descriptors of every layer k >= 2 and the shared tail tables.
template <typename T>
static bool upload(T **dst, const std::vector<T> &v) {
    *dst = nullptr;
    if (v.empty()) return true;
    if (plan_malloc(dst, v.size() * sizeof(T)) != cudaSuccess) {
        *dst = nullptr;
        return false;
    }
    return cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) == cudaSuccess;
}

static slos_status_t build_split_tables(slos_plan_s *p) {
    int h = 0;
    if (!p->tab.enabled || p->space != SLOS_SPACE_FOCK || !split_eligible(p->m, p->n, &h)) return SLOS_OK;
    SplitTables *st = new (std::nothrow) SplitTables();
    if (!st) return fail(SLOS_ERR_OOM, "slos_plan: host allocation failed (split tables)");
    p->split = st;
    st->h = h;
    st->layer.assign(p->n + 1, SplitLayer());
    SplitTailHost tail;
    split_build_tail_host(p->m, h, p->n, tail);
    {
        // tail child rows: local children inside their tail lattices
        const int mL = p->m - h;
        for (int rho = 0; rho < p->n; ++rho) {
            const int64_t cnt = binom_host(rho + mL - 1, mL - 1);
            const int64_t chd = binom_host(rho + 1 + mL - 1, mL - 1);
            for (int64_t i = 0; i < cnt * 8; ++i)
                if ((i % 8) < mL && tail.ctab[(size_t)tail.coff[rho] * 8 + i] >= chd)
                    return fail(SLOS_ERR_INTERNAL, "slos_plan: split tail child out of range");
        }
    }
    memcpy(st->coff, tail.coff, sizeof(st->coff));
    bool ok = upload(&st->tctab, tail.ctab);
    st->bytes = tail.ctab.size() * 2;
    for (int k = 2; ok && k <= p->n; ++k) {
        SplitLayerHost L;
        split_build_layer_host(p->m, h, k, L);
        // the parent blocks must tile layer k-1 in rank order, and every
        // child block the kernel reads through them must lie inside layer k
        const int mL = p->m - h;
        auto tail_size = [&](int rho) { return rho < 0 ? (int64_t)0 : binom_host(rho + mL - 1, mL - 1); };
        int64_t next = 0;
        for (size_t b = 0; b < L.bdesc.size() / 4; ++b) {
            const int64_t base = L.bdesc[4 * b], size = L.bdesc[4 * b + 1], lc = L.bdesc[4 * b + 2];
            const int rho = L.bdesc[4 * b + 3];
            if (base != next || lc + tail_size(rho + 1) > p->F[k])
                return fail(SLOS_ERR_INTERNAL, "slos_plan: split parent blocks out of range");
            next += size;
            for (int j = 0; j < h; ++j)
                if ((int64_t)L.bhead[(size_t)b * kSplitMaxHead + j] + size > p->F[k])
                    return fail(SLOS_ERR_INTERNAL, "slos_plan: split head-child block out of range");
        }
        if (next != p->F[k - 1]) return fail(SLOS_ERR_INTERNAL, "slos_plan: split parent blocks do not cover the layer");
        SplitLayer &D = st->layer[k];
        D.nbblk = (int)(L.bdesc.size() / 4);
        std::vector<int4> bd(D.nbblk);
        memcpy(bd.data(), L.bdesc.data(), L.bdesc.size() * 4);
        ok = upload(&D.bdesc, bd) && upload(&D.bhead, L.bhead) && upload(&D.bchunk, L.bchunk);
        st->bytes += (L.bdesc.size() + L.bhead.size() + L.bchunk.size()) * 4;
    }
    if (!ok) return fail(SLOS_ERR_OOM, "slos_plan: cannot allocate or upload the split-lattice tables");
    return SLOS_OK;
}

// Sorted on-chip layout (tables.h, FusedLayer) from the plan's slot tables.
// Returns false (nothing kept) on an allocation failure.
static bool build_fused_tables(slos_plan_s *p) {
    const int n = p->n;
    std::vector<std::vector<int32_t>> pos(n + 1);
    pos[0].assign(1, 0);
    std::vector<float> wnat(p->F[n]);
    if (cudaMemcpy(wnat.data(), p->tab.w, wnat.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
    p->tab.fused.assign(n + 1, FusedLayer());
    for (int k = 1; k <= n; ++k) {
        const int64_t Fk = p->F[k];
        const int kw = p->tab.layer[k].kw;
        std::vector<uint32_t> nat((size_t)Fk * kw);
        if (cudaMemcpy(nat.data(), p->tab.layer[k].slots, nat.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            return false;
        std::vector<int> occ(Fk, 0);
        int qmax = 0;
        for (int64_t c = 0; c < Fk; ++c) {
            while (occ[c] < kw && nat[(size_t)c * kw + occ[c]] != kSlotEmpty) ++occ[c];
            qmax = std::max(qmax, occ[c]);
        }
        pos[k].assign(Fk, -1);
        std::vector<uint32_t> rows, blk;
        std::vector<int32_t> id;
        std::vector<float> wf;
        int fpad = 0;
        // The final layer is sorted within tiles of kFusedOutTile consecutive
        // output indices, so the CTA's warps, which take blocks in order,
        // write one region of each output row at a time and L2 sees whole
        // sectors (sorted over the whole layer, partly written sectors were
        // evicted and re-read: 1.7x the output bytes in DRAM traffic).
        const int64_t tile = k == n ? kFusedOutTile : Fk;
        for (int64_t t0 = 0; t0 < Fk; t0 += tile) {
            std::vector<std::vector<int64_t>> by_q(qmax + 1);
            for (int64_t c = t0; c < std::min(Fk, t0 + tile); ++c) by_q[occ[c]].push_back(c);
            for (int q = 1; q <= qmax; ++q) {
                const auto &list = by_q[q];
                for (size_t b0 = 0; b0 < list.size(); b0 += 32) {
                    const size_t off = rows.size();
                    blk.push_back((uint32_t)(off << 4) | (uint32_t)q);
                    rows.resize(off + (size_t)q * 32, kSlotEmpty);
                    for (int l = 0; l < 32; ++l) {
                        const int position = fpad + l;
                        int32_t out_id = -1;
                        float wv = 0.f;
                        if (b0 + l < list.size()) {
                            const int64_t c = list[b0 + l];
                            pos[k][c] = position;
                            for (int i = 0; i < q; ++i) {
                                const uint32_t e = nat[(size_t)c * kw + i];
                                const uint32_t pp = (uint32_t)pos[k - 1][e >> 5];
                                rows[off + (size_t)i * 32 + l] = (pp << 5) | (e & 31u);
                            }
                            out_id = (int32_t)c;
                            if (k == n) wv = wnat[c];
                        }
                        if (k == n) {
                            id.push_back(out_id);
                            wf.push_back(wv);
                        }
                    }
                    fpad += 32;
                }
            }
        }
        FusedLayer &FL = p->tab.fused[k];
        FL.nblk = (int)blk.size();
        FL.fpad = fpad;
        if (plan_malloc(&FL.rows, rows.size() * 4) != cudaSuccess || plan_malloc(&FL.blk, blk.size() * 4) != cudaSuccess)
            return false;
        if (!h2d(FL.rows, rows.data(), rows.size() * 4) || !h2d(FL.blk, blk.data(), blk.size() * 4)) return false;
        if (k == n) {
            if (plan_malloc(&p->tab.fused_id, id.size() * 4) != cudaSuccess ||
                plan_malloc(&p->tab.fused_w, wf.size() * 4) != cudaSuccess)
                return false;
            if (!h2d(p->tab.fused_id, id.data(), id.size() * 4) || !h2d(p->tab.fused_w, wf.data(), wf.size() * 4))
                return false;
        }
        if (k > 1) pos[k - 1].clear();
    }
    return true;
}

// On-chip inference forward: PNR table plans whose intermediate layers fit in
// shared memory for at least one instance.  Small plans (up to 24 KB per
// instance): as many instances per CTA as fit in half the limit, two
// 512-thread CTAs per SM.  Larger plans: as many instances as fit in the whole
// limit, one 1024-thread CTA per SM, so each parent-slot row read from L2
// serves more instances (measured on m=12, n=6 and m=10, n=5).
//
// Large plans walk the sorted layout (build_fused_tables) when it still fits
// one instance; small plans walk Fock order (slos_fused.cu gives the timings).
static int fused_ni_for(const int c2[2], int n, size_t limit) {
    int ni = 0;
    for (int q = 1; q <= slos_fused_max_ni(); q *= 2)
        if (slos_fused_smem(q, n, c2) <= limit) ni = q;
    return ni;
}

static void choose_fused(slos_plan_s *p) {
    p->fused_ni = 0;
    p->fused_sorted = false;
    if (!p->tab.enabled || p->det != SLOS_DETECT_PNR) return;
    int64_t cap[2] = {1, 1};
    for (int k = 1; k < p->n; ++k) cap[k & 1] = std::max(cap[k & 1], p->F[k]);
    if (cap[0] + cap[1] > ((int64_t)1 << 24)) return;
    const int c2[2] = {(int)cap[0], (int)cap[1]};
    const bool large = slos_fused_smem(1, p->n, c2) > 24 * 1024;
    const size_t limit = large ? kFusedSmemLimit : kFusedSmemLimit / 2;
    const int ni = fused_ni_for(c2, p->n, limit);
    if (ni == 0) return;
    p->fused_ni = ni;
    p->fused_threads = large ? 1024 : 512;
    p->fused_cap[0] = c2[0];
    p->fused_cap[1] = c2[1];
    if (!large) return;
    if (!build_fused_tables(p)) {
        free_fused_tables(p);
        return;
    }
    int64_t sc[2] = {32, 32};
    for (int k = 1; k < p->n; ++k) sc[k & 1] = std::max<int64_t>(sc[k & 1], p->tab.fused[k].fpad);
    const int s2[2] = {(int)sc[0], (int)sc[1]};
    const int sni = fused_ni_for(s2, p->n, kFusedSmemLimit);
    if (sni == 0) {
        free_fused_tables(p);
        return;
    }
    p->fused_sorted = true;
    p->fused_ni = sni;
    p->fused_cap[0] = s2[0];
    p->fused_cap[1] = s2[1];
}

// ------------------------------------------------------------------ layouts
static int groups_for(int batch) { return (batch + kLanes - 1) / kLanes; }

static int blocks_for(const slos_plan_s *p, int64_t states, int chunk, int NG, int per_sm = 4) {
    const int64_t nchunks = (states + chunk - 1) / chunk;
    const int64_t need = (nchunks + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const int64_t target = std::max<int64_t>(1, (int64_t)p->sm_count * per_sm / std::max(1, NG));
    return (int)std::max<int64_t>(1, std::min(need, std::max<int64_t>(target, 1)));
}

// Table-mode backward: one parent per warp per step, 4-warp blocks, as many
// blocks as the kernel's register budget keeps resident, spread over the groups.
static int bwd_tab_blocks(const slos_plan_s *p, int64_t parents, int NG, bool final_layer) {
    const int64_t need = (parents + kBwdTabWarps - 1) / kBwdTabWarps;
    const int per_sm = bwd_tab_min_blocks(mmax_for(p->m), final_layer);
    const int64_t target = std::max<int64_t>(1, (int64_t)p->sm_count * per_sm / std::max(1, NG));
    return (int)std::max<int64_t>(1, std::min(need, target));
}

// Split-lattice backward: warp runs of kSplitRun parents; the grid fills the
// resident blocks its register budget allows.
static int split_blocks(const slos_plan_s *p, int64_t items, int items_per_block, int NG, int per_sm) {
    const int64_t need = (items + items_per_block - 1) / items_per_block;
    const int64_t target = std::max<int64_t>(1, (int64_t)p->sm_count * per_sm / std::max(1, NG));
    return (int)std::max<int64_t>(1, std::min(need, target));
}
static int64_t split_runs(int64_t states) { return (states + kSplitRun - 1) / kSplitRun; }

constexpr int kChunkStore = 64;
constexpr int kChunkFinal = 32;
constexpr int kChunkBwd = 64;

static Layout make_layout(const slos_plan_s *p, int batch, bool training) {
    Layout L;
    const int n = p->n;
    const int NG = groups_for(batch);
    const size_t row = (size_t)NG * kLanes * sizeof(float2);  // bytes per Fock state
    L.layer.assign(n + 1, SIZE_MAX);
    L.g[0] = L.g[1] = SIZE_MAX;
    L.seedT = SIZE_MAX;
    L.dupart.assign(n + 1, SIZE_MAX);
    L.dpw = SIZE_MAX;
    L.dulayer = SIZE_MAX;
    L.bwd_blocks.assign(n + 1, 0);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align_up(bytes);
        return o;
    };
    L.counters = take(kCounters * sizeof(int));
    if (!training) {
        // ping-pong: layer k in buffer (n-1-k) % 2; a_n only for the
        // threshold pattern sums of plans without tables
        size_t b0 = n >= 2 ? take(row * p->F[n - 1]) : SIZE_MAX;
        size_t b1 = n >= 3 ? take(row * p->F[n - 2]) : SIZE_MAX;
        for (int k = 1; k < n; ++k) L.layer[k] = ((n - 1 - k) % 2 == 0) ? b0 : b1;
        if (p->det == SLOS_DETECT_THRESHOLD && !p->tab.enabled) L.layer[n] = take(row * p->F[n]);
    } else {
        // kept layers + one recompute segment: slot i of a segment holds the
        // i-th non-kept layer above the segment's kept base layer
        std::vector<int64_t> slot_states(n + 1, 0);
        {
            int base = 0;
            for (int k = 1; k < n; ++k) {
                if (p->stored[k]) base = k;
                else slot_states[k - base - 1] = std::max(slot_states[k - base - 1], p->F[k]);
            }
        }
        for (int k = 1; k < n; ++k)
            if (p->stored[k]) L.layer[k] = take(row * p->F[k]);
        L.layer[n] = take(row * p->F[n]);
        std::vector<size_t> slot(n + 1, SIZE_MAX);
        for (int i = 0; i <= n; ++i)
            if (slot_states[i] > 0) slot[i] = take(row * slot_states[i]);
        {
            int base = 0;
            for (int k = 1; k < n; ++k) {
                if (p->stored[k]) base = k;
                else L.layer[k] = slot[k - base - 1];
            }
        }
        if (n >= 2) L.g[0] = take(row * p->F[n - 1]);
        if (n >= 3) L.g[1] = take(row * p->F[n - 2]);
        L.seedT = take(row * p->F[n]);  // c64-sized: enough for either seed kind
        L.dpw = L.seedT;
        for (int k = 1; k <= n; ++k) {
            const int bx = (p->split && k >= 2)
                               ? split_blocks(p, split_runs(p->F[k - 1]), kSplitBwdWarps, NG, kSplitBwdMinBlocks)
                           : p->tab.enabled ? bwd_tab_blocks(p, p->F[k - 1], NG, k == n)
                                            : blocks_for(p, p->F[k - 1], kChunkBwd, NG);
            L.bwd_blocks[k] = bx;
            L.dupart[k] = take((size_t)NG * bx * kLanes * p->m * sizeof(float2));
        }
        L.dulayer = take((size_t)(n + 1) * NG * kLanes * p->m * sizeof(float2));
    }
    L.total = off;
    return L;
}

static void fill_pat_off(const slos_plan_s *p, int *dst) {
    for (int i = 0; i < kMaxPhotons + 2; ++i) dst[i] = p->pat_off[std::min(i, 15)];
}

// dU reduction, in a fixed order.  Pass 1 (grid: layer x group, threads:
// lane x mode): sum the per-block partials of layer k, reading contiguous
// rows.  Pass 2 (thread per dU entry): dU[b][j][i] = sum over the layers k
// whose photon sits in mode i (c_k = i) of the per-layer sums.
struct ReduceArgs {
    const float2 *part[kMaxPhotons + 1];
    int blocks[kMaxPhotons + 1];
    int cols[kMaxPhotons + 1];
    int n, m, B, NG;
    float2 *layer;  // [n + 1][NG][32][m]
    float2 *dU;
};

// grid (layer, group, 32-entry column of [32][m]); warp w sums the partials
// of blocks w, w + 8, ... for its 32 entries, then the 8 warps' sums are added
// in a fixed order
__global__ void dU_layer_sum_kernel(ReduceArgs a) {
    __shared__ float2 part[8][32];
    const int k = blockIdx.x + 1, grp = blockIdx.y;
    const int per = kLanes * a.m;
    const int e = blockIdx.z * 32 + (threadIdx.x & 31);
    const int w = threadIdx.x >> 5;
    const int bx = a.blocks[k];
    const float2 *base = a.part[k] + (int64_t)grp * bx * per;
    float2 s = make_float2(0.f, 0.f);
    if (e < per) {
        for (int blk = w; blk < bx; blk += 8) {
            const float2 v = base[(int64_t)blk * per + e];
            s.x += v.x;
            s.y += v.y;
        }
    }
    part[w][threadIdx.x & 31] = s;
    __syncthreads();
    if (w == 0 && e < per) {
        float2 t = part[0][threadIdx.x];
        for (int q = 1; q < 8; ++q) {
            t.x += part[q][threadIdx.x].x;
            t.y += part[q][threadIdx.x].y;
        }
        a.layer[((int64_t)k * a.NG + grp) * per + e] = t;
    }
}

__global__ void dU_assemble_kernel(ReduceArgs a) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)a.B * a.m * a.m;
    if (tid >= total) return;
    const int i = (int)(tid % a.m);
    const int j = (int)((tid / a.m) % a.m);
    const int b = (int)(tid / ((int64_t)a.m * a.m));
    const int grp = b / kLanes, lane = b % kLanes;
    float2 s = make_float2(0.f, 0.f);
    for (int k = 1; k <= a.n; ++k) {
        if (a.cols[k] != i) continue;
        const float2 v = a.layer[(((int64_t)k * a.NG + grp) * kLanes + lane) * a.m + j];
        s.x += v.x;
        s.y += v.y;
    }
    a.dU[tid] = s;
}

// Device index table (tests): same unrank / occupation / parent arithmetic as
// the SLOS kernels, one thread per state.
template <int MMAX>
__global__ void index_table_kernel(int m, int k, int64_t first, int64_t count, uint8_t *comp, int32_t *par) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int64_t c = first + i;
    const int L = k + m - 1;
    int p[MMAX];
    unrank_bars<MMAX>(c, m, L, p);
    int64_t S = 0;
#pragma unroll
    for (int j = 0; j < MMAX; ++j) {
        if (j < m) {
            const int tj = occupation<MMAX>(j, m, L, p);
            if (comp) comp[i * m + j] = (uint8_t)tj;
            if (par) par[i * m + j] = tj > 0 ? (int32_t)(c - S) : -1;
            if (j < m - 1) S += (int64_t)binom_m1(p[j], m - 2 - j);
        }
    }
}

}  // namespace slos

using namespace slos;

// ==================================================================== ABI
extern "C" {

const char *slos_last_error(void) { return g_last_error.c_str(); }
const char *slos_version(void) { return "libslos 0.1 (sm_103a)"; }

static slos_status_t check_mesh(const slos_mesh_desc_t *d, int batch) {
    if (!d) return fail(SLOS_ERR_INVALID_ARG, "mesh desc is NULL");
    if (d->m < 2 || d->m > kMaxModes) return fail(SLOS_ERR_UNSUPPORTED, "mesh: m must be in [2, 24]");
    if (d->n_data < 0 || d->n_data > d->m) return fail(SLOS_ERR_INVALID_ARG, "mesh: n_data must be in [0, m]");
    if (d->data_col < 0 || d->data_col > d->m) return fail(SLOS_ERR_INVALID_ARG, "mesh: data_col must be in [0, m]");
    if (batch < 0) return fail(SLOS_ERR_INVALID_ARG, "mesh: negative batch");
    return SLOS_OK;
}

static slos_status_t mesh_forward_impl(const slos_mesh_desc_t *desc, const float *theta, int64_t theta_stride_b,
                                       const float *data, int64_t data_stride_b, const float *w, int batch, void *U,
                                       void *stream) {
    slos_status_t st = check_mesh(desc, batch);
    if (st != SLOS_OK) return st;
    if (batch == 0) return SLOS_OK;
    if (!theta || !U) return fail(SLOS_ERR_INVALID_ARG, "mesh_unitary: NULL theta or U");
    if (desc->n_data > 0 && !data) return fail(SLOS_ERR_INVALID_ARG, "mesh_unitary: NULL data with n_data > 0");
    MeshArgs a;
    a.theta = theta;
    a.theta_stride = theta_stride_b;
    a.data = desc->n_data > 0 ? data : nullptr;
    a.data_stride = data_stride_b;
    a.data_w = desc->n_data > 0 ? w : nullptr;
    a.U = reinterpret_cast<float2 *>(U);
    a.m = desc->m;
    a.n_data = desc->n_data;
    a.data_col = desc->data_col;
    a.B = batch;
    {
        ProfScope ps("mesh_fwd", (double)batch * 8.0 * desc->m * desc->m, (cudaStream_t)stream);
        SLOS_CUDA(mesh_forward_launch(a, (cudaStream_t)stream));
    }
    return SLOS_OK;
}

slos_status_t mesh_unitary(const slos_mesh_desc_t *desc, const float *theta, int64_t theta_stride_b,
                           const float *data, int64_t data_stride_b, int batch, void *U, void *stream) {
    return mesh_forward_impl(desc, theta, theta_stride_b, data, data_stride_b, nullptr, batch, U, stream);
}

slos_status_t mesh_unitary_weighted(const slos_mesh_desc_t *desc, const float *theta, int64_t theta_stride_b,
                                    const float *x, int64_t x_stride_b, const float *w, int batch, void *U,
                                    void *stream) {
    if (desc && desc->n_data > 0 && !w) return fail(SLOS_ERR_INVALID_ARG, "mesh_unitary_weighted: NULL w");
    return mesh_forward_impl(desc, theta, theta_stride_b, x, x_stride_b, w, batch, U, stream);
}

slos_status_t mesh_unitary_backward_workspace(const slos_mesh_desc_t *desc, int batch, int64_t theta_stride_b,
                                              size_t *bytes) {
    slos_status_t st = check_mesh(desc, batch);
    if (st != SLOS_OK) return st;
    if (!bytes) return fail(SLOS_ERR_INVALID_ARG, "NULL bytes");
    *bytes = theta_stride_b == 0 ? (size_t)batch * desc->m * (desc->m - 1) * sizeof(float) : 0;
    return SLOS_OK;
}

static slos_status_t mesh_backward_impl(const slos_mesh_desc_t *desc, const float *theta, int64_t theta_stride_b,
                                        const float *data, int64_t data_stride_b, const float *w, int batch,
                                        const void *dU, float *dtheta, float *ddata, float *dw, void *workspace,
                                        size_t workspace_bytes, void *stream) {
    slos_status_t st = check_mesh(desc, batch);
    if (st != SLOS_OK) return st;
    const int m = desc->m;
    const int P = m * (m - 1);
    if (batch == 0) {
        if (theta_stride_b == 0 && dtheta) SLOS_CUDA(cudaMemsetAsync(dtheta, 0, P * sizeof(float), (cudaStream_t)stream));
        return SLOS_OK;
    }
    if (!theta || !dU || !dtheta) return fail(SLOS_ERR_INVALID_ARG, "mesh_unitary_backward: NULL pointer");
    if (desc->n_data > 0 && (!data || !ddata))
        return fail(SLOS_ERR_INVALID_ARG, "mesh_unitary_backward: NULL data/ddata with n_data > 0");
    size_t need = 0;
    mesh_unitary_backward_workspace(desc, batch, theta_stride_b, &need);
    if (workspace_bytes < need || (need > 0 && !workspace))
        return fail(SLOS_ERR_INVALID_ARG, "mesh_unitary_backward: workspace too small");
    MeshBwdArgs a;
    a.theta = theta;
    a.theta_stride = theta_stride_b;
    a.data = desc->n_data > 0 ? data : nullptr;
    a.data_stride = data_stride_b;
    a.data_w = desc->n_data > 0 ? w : nullptr;
    a.dw = desc->n_data > 0 ? dw : nullptr;
    a.dU = reinterpret_cast<const float2 *>(dU);
    a.dtheta = theta_stride_b == 0 ? reinterpret_cast<float *>(workspace) : dtheta;
    a.dtheta_stride = P;
    a.ddata = ddata;
    a.m = m;
    a.n_data = desc->n_data;
    a.data_col = desc->data_col;
    a.B = batch;
    {
        ProfScope ps("mesh_bwd", (double)batch * (8.0 * m * m + 4.0 * P), (cudaStream_t)stream);
        SLOS_CUDA(mesh_backward_launch(a, theta_stride_b == 0 ? dtheta : nullptr, (cudaStream_t)stream));
    }
    return SLOS_OK;
}

slos_status_t mesh_unitary_backward(const slos_mesh_desc_t *desc, const float *theta, int64_t theta_stride_b,
                                    const float *data, int64_t data_stride_b, int batch, const void *dU,
                                    float *dtheta, float *ddata, void *workspace, size_t workspace_bytes,
                                    void *stream) {
    return mesh_backward_impl(desc, theta, theta_stride_b, data, data_stride_b, nullptr, batch, dU, dtheta, ddata,
                              nullptr, workspace, workspace_bytes, stream);
}

slos_status_t mesh_unitary_weighted_backward(const slos_mesh_desc_t *desc, const float *theta, int64_t theta_stride_b,
                                             const float *x, int64_t x_stride_b, const float *w, int batch,
                                             const void *dU, float *dtheta, float *dx, float *dw, void *workspace,
                                             size_t workspace_bytes, void *stream) {
    if (desc && desc->n_data > 0 && !w) return fail(SLOS_ERR_INVALID_ARG, "mesh_unitary_weighted_backward: NULL w");
    return mesh_backward_impl(desc, theta, theta_stride_b, x, x_stride_b, w, batch, dU, dtheta, dx, dw, workspace,
                              workspace_bytes, stream);
}

slos_status_t mesh_sum_rows(const float *rows, int batch, int width, float *out, void *stream) {
    if (batch < 0 || width < 0) return fail(SLOS_ERR_INVALID_ARG, "mesh_sum_rows: negative size");
    if (width == 0) return SLOS_OK;
    if (!out || (batch > 0 && !rows)) return fail(SLOS_ERR_INVALID_ARG, "mesh_sum_rows: NULL pointer");
    cudaStream_t s = (cudaStream_t)stream;
    ProfScope ps("mesh_sum_rows", 4.0 * ((double)batch + 1.0) * width, s);
    SLOS_CUDA(mesh_sum_rows_launch(rows, batch, width, out, s));
    return SLOS_OK;
}

slos_status_t slos_plan(int m, int n, const int *input_state, slos_detection_t detection, size_t mem_budget_bytes,
                        slos_plan_t *out) {
    return slos_plan_space(m, n, input_state, detection, SLOS_SPACE_FOCK, mem_budget_bytes, out);
}

slos_status_t slos_plan_space(int m, int n, const int *input_state, slos_detection_t detection, slos_space_t space,
                              size_t mem_budget_bytes, slos_plan_t *out) {
    if (!out) return fail(SLOS_ERR_INVALID_ARG, "slos_plan: NULL out");
    *out = nullptr;
    if (!input_state) return fail(SLOS_ERR_INVALID_ARG, "slos_plan: NULL input_state");
    if (m < 2 || m > kMaxModes) return fail(SLOS_ERR_UNSUPPORTED, "slos_plan: m must be in [2, 24]");
    if (n < 1 || n > kMaxPhotons) return fail(SLOS_ERR_UNSUPPORTED, "slos_plan: n must be in [1, 12]");
    if (detection != SLOS_DETECT_PNR && detection != SLOS_DETECT_THRESHOLD)
        return fail(SLOS_ERR_INVALID_ARG, "slos_plan: unknown detection");
    int tot = 0;
    for (int i = 0; i < m; ++i) {
        if (input_state[i] < 0) return fail(SLOS_ERR_INVALID_ARG, "slos_plan: negative occupation");
        tot += input_state[i];
    }
    if (tot != n) return fail(SLOS_ERR_INVALID_ARG, "slos_plan: input_state does not hold n photons");
    if (space != SLOS_SPACE_FOCK && space != SLOS_SPACE_UNBUNCHED)
        return fail(SLOS_ERR_INVALID_ARG, "slos_plan_space: unknown computation space");
    const bool unb = space == SLOS_SPACE_UNBUNCHED;
    if (unb && detection != SLOS_DETECT_PNR)
        return fail(SLOS_ERR_UNSUPPORTED, "slos_plan_space: the collision-free space takes PNR detection");
    if (unb && n > m)
        return fail(SLOS_ERR_INVALID_ARG, "slos_plan_space: no collision-free state holds more photons than modes");
    if (!unb && binom_host(m + n - 1, n) >= (int64_t)1 << 31)
        return fail(SLOS_ERR_UNSUPPORTED, "slos_plan: Fock space too large (>= 2^31 states)");
    slos_plan_s *p = new (std::nothrow) slos_plan_s();
    if (!p) return fail(SLOS_ERR_OOM, "slos_plan: host allocation failed");
    p->kind = 0;
    p->m = m;
    p->n = n;
    p->s.assign(input_state, input_state + m);
    for (int i = 0; i < m; ++i)
        for (int q = 0; q < input_state[i]; ++q) p->cols.push_back(i);
    p->det = detection;
    p->space = (int)space;
    p->F.resize(n + 1);
    for (int k = 0; k <= n; ++k) p->F[k] = unb ? binom_host(m, k) : binom_host(m + k - 1, k);
    double sf = 1.0;
    for (int i = 0; i < m; ++i)
        for (int q = 2; q <= input_state[i]; ++q) sf *= q;
    p->inv_sfact = (float)(1.0 / sf);
    memset(p->pat_off, 0, sizeof(p->pat_off));
    {
        int64_t acc = 0;
        for (int i = 1; i <= std::min(n, m) && i < 16; ++i) {
            p->pat_off[i] = (int)acc;
            acc += binom_host(m, i);
        }
        p->K = detection == SLOS_DETECT_PNR ? p->F[n] : acc;
    }
    // checkpoint schedule: keep layers k = n-1, n-1-s, n-1-2s, ... with the
    // smallest s whose kept layers plus one recompute segment fit the budget
    // (a_n is always kept: it seeds the backward pass)
    auto bytes_for = [&](int s) {
        int64_t states = 0, seg = 0, seg_max = 0;
        for (int k = 1; k < n; ++k) {
            if ((n - 1 - k) % s == 0) {
                states += p->F[k];
                seg = 0;
            } else {
                seg += p->F[k];
                seg_max = std::max(seg_max, seg);
            }
        }
        return (size_t)(states + seg_max) * sizeof(float2);
    };
    int s = 1;
    if (mem_budget_bytes > 0) {
        while (s < n && bytes_for(s) > mem_budget_bytes) ++s;
    }
    p->stride = s;
    p->stored.assign(n + 1, 0);
    for (int k = 1; k < n; ++k) p->stored[k] = ((n - 1 - k) % s == 0);
    p->stored[n] = 1;
    p->batched = nullptr;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        return fail(SLOS_ERR_CUDA, "slos_plan: no CUDA device");
    }
    cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device);
    if (p->sm_count <= 0) p->sm_count = 148;
    cudaError_t e = init_device_once(p->device);
    if (e != cudaSuccess) {
        delete p;
        return fail(SLOS_ERR_CUDA, std::string("slos_plan: kernel attributes: ") + cudaGetErrorString(e));
    }
    if (plan_malloc(&p->d_status, 64) != cudaSuccess) {
        delete p;
        return fail(SLOS_ERR_OOM, "slos_plan: cannot allocate the status word");
    }
    if (cudaMemset(p->d_status, 0, 64) != cudaSuccess) {
        cudaFree(p->d_status);
        delete p;
        return fail(SLOS_ERR_CUDA, "slos_plan: cannot clear the status word");
    }
    slos_status_t tst = build_tables(p);
    if (tst != SLOS_OK) {
        cudaFree(p->d_status);
        delete p;
        return tst;
    }
    tst = build_split_tables(p);
    if (tst != SLOS_OK) {
        free_tables(p);
        cudaFree(p->d_status);
        delete p;
        return tst;
    }
    choose_fused(p);
    // the small leading layers on chip (Fock-space table plans: the child tables have no holes)
    p->prefix_L = (p->tab.enabled && p->space == SLOS_SPACE_FOCK) ? slos_prefix_layers(p->m, p->n, p->F.data()) : 0;
    tst = build_encode_tables(p);
    if (tst != SLOS_OK) {
        free_tables(p);
        cudaFree(p->d_status);
        delete p;
        return tst;
    }
    *out = p;
    return SLOS_OK;
}

slos_status_t slos_plan_query(slos_plan_t p, int64_t *n_outputs, int64_t *fock_dim, int *checkpoint_stride) {
    if (!p || p->kind != 0) return fail(SLOS_ERR_INVALID_ARG, "slos_plan_query: not a single-shape plan");
    if (n_outputs) *n_outputs = p->K;
    if (fock_dim) *fock_dim = p->F[p->n];
    if (checkpoint_stride) *checkpoint_stride = p->stride;
    return SLOS_OK;
}

slos_status_t slos_workspace_bytes(slos_plan_t p, int batch, int training, size_t *bytes) {
    if (!p || p->kind != 0 || !bytes || batch < 0)
        return fail(SLOS_ERR_INVALID_ARG, "slos_workspace_bytes: bad argument");
    *bytes = batch == 0 ? 0 : make_layout(p, batch, training != 0).total;
    return SLOS_OK;
}

// Backward seed from the plan's weight table (plans whose outputs are not
// enumerated by the Fock index arithmetic, i.e. the collision-free space):
// shared seed: dpw[t] = 2 w_t dout[t]; per instance: seedT[g][t][lane] =
// 2 w_t dout[b][t] (probabilities) or sqrt(w_t) dout[b][t] (amplitudes).
struct SeedTabArgs {
    const void *dout;
    int64_t stride;
    void *outT;
    const float *w;
    int64_t Fn;
    int B, kind, bcast;  // kind: 0 probabilities, 1 amplitudes
};

__global__ void seed_table_kernel(SeedTabArgs a) {
    if (a.bcast) {
        const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        if (c < a.Fn) reinterpret_cast<float *>(a.outT)[c] = 2.f * a.w[c] * reinterpret_cast<const float *>(a.dout)[c];
        return;
    }
    const int lane = threadIdx.x & 31;
    const int grp = blockIdx.y;
    const int b = grp * kLanes + lane;
    const bool valid = b < a.B;
    const int64_t wpb = blockDim.x >> 5;
    for (int64_t c = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); c < a.Fn; c += (int64_t)gridDim.x * wpb) {
        const size_t o = ((size_t)grp * a.Fn + c) * kLanes + lane;
        const float wc = __ldg(a.w + c);
        if (a.kind == 0) {
            const float v = valid ? reinterpret_cast<const float *>(a.dout)[(int64_t)b * a.stride + c] : 0.f;
            reinterpret_cast<float *>(a.outT)[o] = 2.f * wc * v;
        } else {
            const float2 v = valid ? reinterpret_cast<const float2 *>(a.dout)[(int64_t)b * a.stride + c]
                                   : make_float2(0.f, 0.f);
            reinterpret_cast<float2 *>(a.outT)[o] = cscale(v, sqrtf(wc));
        }
    }
}

static slos_status_t launch_layer_fwd(slos_plan_s *p, const Layout &Ly, char *ws, const float2 *U, int batch, int k,
                                      int epi, bool save, void *out, cudaStream_t s, bool recompute = false) {
    int *counter = reinterpret_cast<int *>(ws + Ly.counters) + (recompute ? kCtrRecompute + k : k);
    const int NG = groups_for(batch);
    FwdArgs a;
    memset(&a, 0, sizeof(a));
    a.prev = k >= 2 ? reinterpret_cast<const float2 *>(ws + Ly.layer[k - 1]) : nullptr;
    a.next = (epi == EPI_STORE || save) ? reinterpret_cast<float2 *>(ws + Ly.layer[k]) : nullptr;
    a.U = U;
    a.out = out;
    a.Fk = p->F[k];
    a.Fprev = p->F[k - 1];
    a.K = p->K;
    a.m = p->m;
    a.k = k;
    a.col = p->cols[k - 1];
    a.B = batch;
    a.NG = NG;
    a.chunk = epi == EPI_STORE ? kChunkStore : kChunkFinal;
    a.inv_sfact = p->inv_sfact;
    a.status = p->d_status;
    const int bx = blocks_for(p, a.Fk, a.chunk, NG);
    // layered-model bytes: read a_{k-1}, write a_k and/or the output
    double bytes = (k >= 2 ? 8.0 * a.Fprev : 0.0);
    const char *name = recompute ? "slos_fwd_recompute" : "slos_fwd_layer";
    if (epi == EPI_STORE) {
        bytes += 8.0 * a.Fk;
    } else {
        name = "slos_fwd_final";
        bytes += (epi == EPI_AMPS ? 8.0 : 4.0) * p->K + (save ? 8.0 * a.Fk : 0.0);
    }
    ProfScope ps(name, bytes * batch, s);
    if (p->tab.enabled) {
        TabArgs t{};
        t.slots = p->tab.layer[k].slots;
        t.kw = p->tab.layer[k].kw;
        t.w = p->tab.w;
        t.work = counter;
        t.nseg = 0;
        if (epi == EPI_THRESH) {
            // the final layer in pattern-grouped list order (tables.h)
            t.w = p->tab.lw;
            t.lrank = p->tab.lrank;
            t.lpat = p->tab.lpat;
            t.lseg = p->tab.lseg;
            t.nseg = p->tab.nseg;
        }
        // warp items: one chunk of consecutive states (threshold: one run of
        // whole patterns) of a group pair
        const int64_t chunks = epi == EPI_THRESH ? t.nseg : (a.Fk + slos_pair_chunk() - 1) / slos_pair_chunk();
        const int64_t items = chunks * ((NG + 1) / 2);
        const int64_t blocks = (items + slos_pair_warps() - 1) / slos_pair_warps();
        const int res = slos_pair_resident_blocks(p->m);
        const int bps = p->tune_fwd_bps > 0 ? std::min(p->tune_fwd_bps, res) : res;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)p->sm_count * bps));
        SLOS_CUDA(slos_launch_fwd_pair(a, t, epi, save, grid, s));
    } else {
        SLOS_CUDA(launch_fwd(p->m, a, epi, save, bx, s));
    }
    return SLOS_OK;
}

// Prefix depth in use: the tuned one, else the largest that fits.
static int prefix_layers(const slos_plan_s *p) { return p->tune_prefix_L >= 0 ? p->tune_prefix_L : p->prefix_L; }

static PrefixArgs prefix_args(const slos_plan_s *p, const float2 *U, int batch) {
    PrefixArgs pa;
    memset(&pa, 0, sizeof(pa));
    const int L = prefix_layers(p);
    pa.U = U;
    for (int k = 0; k <= L; ++k) pa.F[k] = (int)p->F[k];
    for (int k = 1; k <= L; ++k) {
        pa.slots[k] = p->tab.layer[k].slots;
        pa.kw[k] = p->tab.layer[k].kw;
        pa.ctab[k] = p->tab.layer[k].ctab;
        pa.cols[k - 1] = p->cols[k - 1];
    }
    pa.cap[0] = pa.cap[1] = 1;
    for (int k = 1; k <= L; ++k) pa.cap[k & 1] = std::max(pa.cap[k & 1], (int)p->F[k]);
    for (int k = 0; k < L; ++k) pa.asum += (int)p->F[k];
    pa.m = p->m;
    pa.L = L;
    pa.B = batch;
    pa.NI = slos_prefix_ni(p->m, L, p->F.data(), batch, p->sm_count);
    if (p->tune_prefix_ni > 0 && slos_prefix_bwd_smem(p->tune_prefix_ni, L, p->F.data()) <= kPrefixSmemLimit)
        pa.NI = p->tune_prefix_ni;
    return pa;
}

// Layers 1..prefix_L in one on-chip launch; writes layer k to the workspace
// when bit k of `want` is set.
static slos_status_t launch_prefix_fwd(const slos_plan_s *p, const Layout &Ly, char *ws, const float2 *U, int batch,
                                       uint32_t want, const char *name, cudaStream_t s) {
    PrefixArgs pa = prefix_args(p, U, batch);
    double bytes = 8.0 * p->m * p->m;
    for (int k = 1; k <= pa.L; ++k)
        if ((want >> k) & 1u) {
            pa.out[k] = reinterpret_cast<float2 *>(ws + Ly.layer[k]);
            bytes += 8.0 * p->F[k];
        }
    ProfScope ps(name, bytes * batch, s);
    SLOS_CUDA(slos_launch_prefix_fwd(pa, s));
    return SLOS_OK;
}

slos_status_t slos_forward(slos_plan_t p, const void *U, int batch, slos_output_t output, void *out,
                           int save_for_backward, void *workspace, size_t workspace_bytes, void *stream) {
    if (!p || p->kind != 0) return fail(SLOS_ERR_INVALID_ARG, "slos_forward: not a single-shape plan");
    if (batch < 0) return fail(SLOS_ERR_INVALID_ARG, "slos_forward: negative batch");
    if (output != SLOS_OUT_PROBS && output != SLOS_OUT_AMPS) return fail(SLOS_ERR_INVALID_ARG, "slos_forward: bad output");
    if (output == SLOS_OUT_AMPS && p->det != SLOS_DETECT_PNR)
        return fail(SLOS_ERR_INVALID_ARG, "slos_forward: amplitudes are only defined before detection (use PNR plan)");
    if (batch == 0) return SLOS_OK;
    if (!U || !out) return fail(SLOS_ERR_INVALID_ARG, "slos_forward: NULL U or out");
    const bool save = save_for_backward != 0;
    {
        slos_status_t st = check_stream(p, (cudaStream_t)stream, "slos_forward");
        if (st != SLOS_OK) return st;
    }
    const Layout Ly = make_layout(p, batch, save);
    if (workspace_bytes < Ly.total || (Ly.total > 0 && !workspace))
        return fail(SLOS_ERR_INVALID_ARG, "slos_forward: workspace too small (" + std::to_string(workspace_bytes) +
                                               " < " + std::to_string(Ly.total) + ")");
    if (reinterpret_cast<uintptr_t>(workspace) % kAlign != 0)
        return fail(SLOS_ERR_INVALID_ARG, "slos_forward: workspace must be 256-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    char *ws = reinterpret_cast<char *>(workspace);
    const float2 *Ud = reinterpret_cast<const float2 *>(U);
    const int n = p->n;
    if (!save && p->fused_ni > 0) {
        // whole plan on chip: only U in and the outputs out
        FusedArgs fa;
        memset(&fa, 0, sizeof(fa));
        fa.U = Ud;
        fa.out = out;
        fa.sorted = p->fused_sorted ? 1 : 0;
        fa.w = p->tab.w;
        fa.ws = p->tab.fused_w;
        fa.id = p->tab.fused_id;
        for (int k = 1; k <= n; ++k) {
            fa.slots[k] = p->tab.layer[k].slots;
            fa.kw[k] = p->tab.layer[k].kw;
            fa.F[k] = (int)p->F[k];
            if (p->fused_sorted) {
                fa.rows[k] = p->tab.fused[k].rows;
                fa.blk[k] = p->tab.fused[k].blk;
                fa.nblk[k] = p->tab.fused[k].nblk;
            }
            fa.cols[k - 1] = p->cols[k - 1];
        }
        fa.F[0] = 1;
        fa.cap[0] = p->fused_cap[0];
        fa.cap[1] = p->fused_cap[1];
        fa.m = p->m;
        fa.n = n;
        fa.B = batch;
        fa.K = (int)p->K;
        fa.NI = p->fused_ni;
        fa.threads = p->fused_threads;
        const double bytes = (double)batch * (8.0 * p->m * p->m + (output == SLOS_OUT_AMPS ? 8.0 : 4.0) * p->K);
        ProfScope ps("slos_fwd_fused", bytes, s);
        SLOS_CUDA(slos_launch_fused(fa, output == SLOS_OUT_AMPS ? EPI_AMPS : EPI_PROBS, s));
        return SLOS_OK;
    }
    SLOS_CUDA(cudaMemsetAsync(ws + Ly.counters, 0, kCounters * sizeof(int), s));
    int k0 = 1;
    if (prefix_layers(p) >= 2) {
        // kept layers of the prefix and its last layer (which layer L + 1 reads)
        const int L = prefix_layers(p);
        uint32_t want = 1u << L;
        for (int k = 1; k < L; ++k)
            if (save && p->stored[k]) want |= 1u << k;
        slos_status_t st = launch_prefix_fwd(p, Ly, ws, Ud, batch, want, "slos_fwd_prefix", s);
        if (st != SLOS_OK) return st;
        k0 = L + 1;
    }
    for (int k = k0; k < n; ++k) {
        slos_status_t st = launch_layer_fwd(p, Ly, ws, Ud, batch, k, EPI_STORE, true, nullptr, s);
        if (st != SLOS_OK) return st;
    }
    if (p->det != SLOS_DETECT_THRESHOLD)
        return launch_layer_fwd(p, Ly, ws, Ud, batch, n, output == SLOS_OUT_AMPS ? EPI_AMPS : EPI_PROBS, save, out, s);
    // threshold: each pattern summed in a fixed order by one warp, during the
    // final layer's walk (tables) or from the stored a_n (no tables)
    if (p->tab.enabled) return launch_layer_fwd(p, Ly, ws, Ud, batch, n, EPI_THRESH, save, out, s);
    slos_status_t st = launch_layer_fwd(p, Ly, ws, Ud, batch, n, EPI_STORE, true, nullptr, s);
    if (st != SLOS_OK) return st;
    ThreshArgs ta;
    memset(&ta, 0, sizeof(ta));
    ta.an = reinterpret_cast<const float2 *>(ws + Ly.layer[n]);
    ta.out = reinterpret_cast<float *>(out);
    ta.Fn = p->F[n];
    ta.K = p->K;
    ta.m = p->m;
    ta.n = n;
    ta.B = batch;
    ta.NG = groups_for(batch);
    ta.jmax = std::min(n, p->m);
    ta.inv_sfact = p->inv_sfact;
    ta.status = p->d_status;
    ProfScope ps("slos_thresh_sum", (8.0 * p->F[n] + 4.0 * p->K) * batch, s);
    SLOS_CUDA(slos_launch_thresh_sum(ta, s));
    return SLOS_OK;
}

slos_status_t slos_backward(slos_plan_t p, const void *U, int batch, slos_output_t output, const void *dout,
                            int64_t dout_stride_b, void *dU, void *workspace, size_t workspace_bytes, void *stream) {
    if (!p || p->kind != 0) return fail(SLOS_ERR_INVALID_ARG, "slos_backward: not a single-shape plan");
    if (batch < 0) return fail(SLOS_ERR_INVALID_ARG, "slos_backward: negative batch");
    if (output == SLOS_OUT_AMPS && p->det != SLOS_DETECT_PNR)
        return fail(SLOS_ERR_INVALID_ARG, "slos_backward: amplitudes need a PNR plan");
    if (batch == 0) return SLOS_OK;
    if (!U || !dout || !dU) return fail(SLOS_ERR_INVALID_ARG, "slos_backward: NULL pointer");
    if (dout_stride_b < 0) return fail(SLOS_ERR_INVALID_ARG, "slos_backward: negative dout stride");
    {
        slos_status_t st = check_stream(p, (cudaStream_t)stream, "slos_backward");
        if (st != SLOS_OK) return st;
    }
    const Layout Ly = make_layout(p, batch, true);
    if (workspace_bytes < Ly.total || !workspace)
        return fail(SLOS_ERR_INVALID_ARG, "slos_backward: workspace too small (need the training size)");
    if (reinterpret_cast<uintptr_t>(workspace) % kAlign != 0)
        return fail(SLOS_ERR_INVALID_ARG, "slos_backward: workspace must be 256-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    char *ws = reinterpret_cast<char *>(workspace);
    const float2 *Ud = reinterpret_cast<const float2 *>(U);
    const int n = p->n, m = p->m;
    const int NG = groups_for(batch);
    SLOS_CUDA(cudaMemsetAsync(ws + Ly.counters, 0, kCounters * sizeof(int), s));

    // seed: the factorial weights are folded in here (see Seed)
    int seed;
    const void *seed_ptr;
    {
        PrepArgs pa;
        memset(&pa, 0, sizeof(pa));
        pa.dout = dout;
        pa.stride = dout_stride_b;
        pa.Fn = p->F[n];
        pa.m = m;
        pa.n = n;
        pa.B = batch;
        pa.NG = NG;
        pa.chunk = kChunkStore;
        pa.inv_sfact = p->inv_sfact;
        pa.kind = output == SLOS_OUT_AMPS ? 1 : (p->det == SLOS_DETECT_THRESHOLD ? 2 : 0);
        fill_pat_off(p, pa.pat_off);
        const bool bcast = dout_stride_b == 0 && pa.kind != 1;
        pa.outT = ws + (bcast ? Ly.dpw : Ly.seedT);
        ProfScope ps("slos_seed_prep", bcast ? 8.0 * p->F[n]
                                            : (double)batch * ((pa.kind == 1 ? 16.0 : 8.0) * p->F[n]), s);
        // plans with tables read the final-layer weights prod t! / prod s! from
        // the plan's table instead of unranking every state (threshold plans
        // also need the pattern of each state and keep the arithmetic kernel)
        if (p->space == SLOS_SPACE_UNBUNCHED || (p->tab.enabled && pa.kind != 2)) {
            SeedTabArgs sa;
            sa.dout = dout;
            sa.stride = dout_stride_b;
            sa.outT = pa.outT;
            sa.w = p->tab.w;
            sa.Fn = p->F[n];
            sa.B = batch;
            sa.kind = pa.kind;
            sa.bcast = bcast ? 1 : 0;
            if (bcast) {
                seed_table_kernel<<<(unsigned)((p->F[n] + 255) / 256), 256, 0, s>>>(sa);
            } else {
                dim3 grid((unsigned)std::min<int64_t>((p->F[n] + 7) / 8, (int64_t)p->sm_count * 8), NG);
                seed_table_kernel<<<grid, 256, 0, s>>>(sa);
            }
            SLOS_CUDA(cudaGetLastError());
        } else {
            SLOS_CUDA(launch_prep(m, pa, blocks_for(p, pa.Fn, pa.chunk, NG), bcast, s));
        }
        seed = bcast ? SEED_BCAST : (pa.kind == 1 ? SEED_AMPS_T : SEED_T);
        seed_ptr = pa.outT;
    }

    int have_base = -1;  // segment currently recomputed (its kept base layer)
    ReduceArgs ra;
    memset(&ra, 0, sizeof(ra));
    const int L = prefix_layers(p);
    for (int k = n; k >= 1; --k) {
        const int kp = k - 1;
        int bx = Ly.bwd_blocks[k];  // CTAs per group of this layer's launch (dU partial rows)
        if (L >= 2 && k <= L) {
            // layers L..1 on chip: a_1..a_{L-1} recomputed, G_L read, one dU row per layer
            PrefixArgs pa = prefix_args(p, Ud, batch);
            pa.GL = reinterpret_cast<const float2 *>(ws + Ly.g[(n - 1 - L) % 2]);
            for (int q = 1; q <= L; ++q) {
                pa.dUpart[q] = reinterpret_cast<float2 *>(ws + Ly.dupart[q]);
                ra.part[q] = pa.dUpart[q];
                ra.blocks[q] = 1;
                ra.cols[q] = p->cols[q - 1];
            }
            ProfScope ps("slos_bwd_prefix", (8.0 * p->F[L] + 8.0 * p->m * p->m) * batch, s);
            SLOS_CUDA(slos_launch_prefix_bwd(pa, s));
            break;
        }
        // an intermediate split layer whose parent layer kp alone was not kept (kp - 1
        // kept, kp + 1 kept): a_kp is formed per parent inside the backward launch from
        // a_{kp-1} instead of being recomputed into the workspace and read back
        const bool fuse_prev = p->split && k >= 2 && k < n && kp > L && kp >= 2 && !p->stored[kp] &&
                               p->stored[kp - 1] && p->stored[kp + 1] && p->tab.layer[kp].kw == 8;
        if (kp >= 1 && !p->stored[kp] && !fuse_prev) {
            int base = kp;
            while (base >= 1 && !p->stored[base]) --base;
            if (base != have_base) {
                int top = kp;
                while (top + 1 < n && !p->stored[top + 1]) ++top;
                if (L >= 2 && top == L) {
                    // the segment ends at the prefix's last layer: only a_L is needed
                    // above the prefix, recomputed on chip from U
                    slos_status_t st = launch_prefix_fwd(p, Ly, ws, Ud, batch, 1u << L, "slos_fwd_recompute", s);
                    if (st != SLOS_OK) return st;
                } else {
                    for (int q = base + 1; q <= top; ++q) {
                        slos_status_t st =
                            launch_layer_fwd(p, Ly, ws, Ud, batch, q, EPI_STORE, true, nullptr, s, true);
                        if (st != SLOS_OK) return st;
                    }
                }
                have_base = base;
            }
        }
        BwdArgs a;
        memset(&a, 0, sizeof(a));
        a.aprev = kp >= 1 ? reinterpret_cast<const float2 *>(ws + Ly.layer[kp]) : nullptr;
        a.Gk = k < n ? reinterpret_cast<const float2 *>(ws + Ly.g[(n - 1 - k) % 2]) : nullptr;
        a.Gprev = kp >= 1 ? reinterpret_cast<float2 *>(ws + Ly.g[(n - 1 - kp) % 2]) : nullptr;
        a.an = k == n ? reinterpret_cast<const float2 *>(ws + Ly.layer[n]) : nullptr;
        a.seed = seed_ptr;
        a.U = Ud;
        a.dUpart = reinterpret_cast<float2 *>(ws + Ly.dupart[k]);
        a.Fk = p->F[k];
        a.Fprev = p->F[kp];
        a.m = m;
        a.k = k;
        a.col = p->cols[k - 1];
        a.B = batch;
        a.NG = NG;
        a.chunk = kChunkBwd;
        a.inv_sfact = p->inv_sfact;
        {
            // layered-model bytes: read a_{k-1} and G_k (or a_n and the seed), write
            // G_{k-1}; a seed shared by the batch is read once
            double bytes = (kp >= 1 ? 16.0 * a.Fprev : 0.0) + 8.0 * a.Fk;
            double shared = 0.0;
            if (k == n && seed == SEED_T) bytes += 4.0 * a.Fk;
            if (k == n && seed == SEED_BCAST) shared = 4.0 * a.Fk;
            ProfScope ps(k == n ? "slos_bwd_final" : "slos_bwd_layer", bytes * batch + shared, s);
            if (p->split && k >= 2) {
                const SplitTables &st = *p->split;
                const SplitLayer &L = st.layer[k];
                SplitBwdArgs sa;
                memset(&sa, 0, sizeof(sa));
                sa.aprev = a.aprev;
                sa.Gk = a.Gk;
                sa.Gprev = a.Gprev;
                sa.an = a.an;
                sa.seed = a.seed;
                sa.U = Ud;
                sa.dUpart = a.dUpart;
                sa.desc = L.bdesc;
                sa.head = L.bhead;
                sa.chunk = L.bchunk;
                sa.tctab = st.tctab;
                memcpy(sa.coff, st.coff, sizeof(sa.coff));
                sa.Fk = (int)p->F[k];
                sa.Fprev = (int)p->F[kp];
                sa.nruns = (int)split_runs(p->F[kp]);
                sa.m = m;
                sa.col = a.col;
                sa.B = batch;
                sa.status = p->d_status;
                // a tuned grid is never wider than the layout's dU partial rows
                if (p->tune_bwd_bps > 0)
                    bx = std::min(bx, split_blocks(p, sa.nruns, kSplitBwdWarps, NG, p->tune_bwd_bps));
                if (fuse_prev) {
                    sa.pslots = p->tab.layer[kp].slots;
                    sa.pprev = reinterpret_cast<const float2 *>(ws + Ly.layer[kp - 1]);
                    sa.pcol = p->cols[kp - 1];
                    sa.Fpp = (int)p->F[kp - 1];
                }
                SLOS_CUDA(slos_launch_bwd_split(sa, NG, k == n ? seed : SEED_G, st.h, bx, s, fuse_prev));
            } else if (p->tab.enabled)
                SLOS_CUDA(launch_bwd_tab(m, a, p->tab.layer[k].ctab, k == n ? seed : SEED_G, Ly.bwd_blocks[k],
                                         p->space == SLOS_SPACE_UNBUNCHED, s));
            else
                SLOS_CUDA(launch_bwd(m, a, k == n ? seed : SEED_G, Ly.bwd_blocks[k], s));
        }
        ra.part[k] = a.dUpart;
        ra.blocks[k] = bx;
        ra.cols[k] = a.col;
    }
    ra.n = n;
    ra.m = m;
    ra.B = batch;
    ra.NG = NG;
    ra.layer = reinterpret_cast<float2 *>(ws + Ly.dulayer);
    ra.dU = reinterpret_cast<float2 *>(dU);
    const int64_t tot = (int64_t)batch * m * m;
    {
        double bytes = 0.0;
        for (int k = 1; k <= n; ++k) bytes += 8.0 * NG * ra.blocks[k] * kLanes * m;
        ProfScope ps("slos_dU_reduce", bytes + 8.0 * tot, s);
        dU_layer_sum_kernel<<<dim3(n, NG, (kLanes * m + 31) / 32), 256, 0, s>>>(ra);
        SLOS_CUDA(cudaGetLastError());
        count_launch();
        dU_assemble_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(ra);
        SLOS_CUDA(cudaGetLastError());
    }
    return SLOS_OK;
}

// ------------------------------------------------------------------ single-shape autotuner
// Key of a single-shape plan's tuned launch shapes: device, shape and batch.
static std::string tune_key(const slos_plan_s *p, int batch) {
    cudaDeviceProp prop;
    std::string dev = cudaGetDeviceProperties(&prop, p->device) == cudaSuccess ? prop.name : "unknown";
    std::ostringstream k;
    k << dev << "|single:m" << p->m << ",n" << p->n << ",s";
    for (int v : p->s) k << v << ".";
    k << ",det" << (int)p->det << ",space" << p->space << ",stride" << p->stride << ",batch" << batch;
    return k.str();
}

// Integer field `name` of one JSON line of the cache; false when absent.
static bool json_int(const std::string &line, const char *name, int *v) {
    const std::string pat = std::string("\"") + name + "\": ";
    const size_t i = line.find(pat);
    if (i == std::string::npos) return false;
    *v = atoi(line.c_str() + i + pat.size());
    return true;
}

static bool tune_lookup(const char *path, const std::string &key, int out[4]) {
    std::ifstream f(path);
    if (!f) return false;
    std::string line;
    bool found = false;
    const std::string kq = "\"key\": \"" + key + "\"";
    while (std::getline(f, line)) {
        if (line.find(kq) == std::string::npos) continue;
        int v[4];
        if (json_int(line, "prefix_layers", &v[0]) && json_int(line, "prefix_ni", &v[1]) &&
            json_int(line, "fwd_blocks_per_sm", &v[2]) && json_int(line, "bwd_blocks_per_sm", &v[3])) {
            memcpy(out, v, sizeof(v));
            found = true;  // the last entry for the key wins
        }
    }
    return found;
}

static void tune_apply(slos_plan_s *p, const int t[4]) {
    p->tune_prefix_L = t[0];
    p->tune_prefix_ni = t[1];
    p->tune_fwd_bps = t[2];
    p->tune_bwd_bps = t[3];
}

constexpr int kTuneReps = 4;  // timed training pairs per candidate

slos_status_t slos_autotune(slos_plan_t p, const void *U, int batch, void *out, const float *dout_shared, void *dU,
                            void *workspace, size_t workspace_bytes, const char *cache_path, void *stream) {
    if (!p || p->kind != 0) return fail(SLOS_ERR_INVALID_ARG, "slos_autotune: not a single-shape plan");
    if (batch <= 0 || !U || !out || !dout_shared || !dU || !workspace)
        return fail(SLOS_ERR_INVALID_ARG, "slos_autotune: empty batch or NULL pointer");
    const std::string key = tune_key(p, batch);
    int best_t[4] = {-1, 0, 0, 0};
    if (cache_path && tune_lookup(cache_path, key, best_t)) {
        tune_apply(p, best_t);
        return SLOS_OK;
    }
    // candidates: prefix depth (none, or 2..largest), its instances per CTA,
    // and the grid widths of the forward and backward layer launches
    // the default shape first: a candidate replaces it only when it is more
    // than 0.5 % faster, so timing noise does not move the choice
    std::vector<int> Ls;
    for (int L = p->prefix_L; L >= 2; --L) Ls.push_back(L);
    Ls.push_back(0);
    const int res = slos_pair_resident_blocks(p->m);
    const int fwd_opts[] = {res, std::max(1, res - 2)};
    const int bwd_opts[] = {kSplitBwdMinBlocks, kSplitBwdMinBlocks - 1};
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return fail(SLOS_ERR_CUDA, "slos_autotune: cannot create events");
    }
    slos_status_t st = SLOS_OK;
    float best = 1e30f;
    auto run = [&](void) -> slos_status_t {
        slos_status_t r = slos_forward(p, U, batch, SLOS_OUT_PROBS, out, 1, workspace, workspace_bytes, stream);
        if (r != SLOS_OK) return r;
        return slos_backward(p, U, batch, SLOS_OUT_PROBS, dout_shared, 0, dU, workspace, workspace_bytes, stream);
    };
    const int ni_def = slos_prefix_ni(p->m, p->prefix_L, p->F.data(), batch, p->sm_count);
    std::vector<int> nis = {ni_def};  // the default instance count first, then the others
    for (int v : {1, 2, 4})
        if (v != ni_def) nis.push_back(v);
    bool first = true;
    for (int L : Ls) {
        for (int ni : nis) {
            if (L == 0 && ni > 1) continue;
            if (L > 0 && (ni > batch || slos_prefix_bwd_smem(ni, L, p->F.data()) > kPrefixSmemLimit)) continue;
            for (int fb : fwd_opts) {
                for (int bb : bwd_opts) {
                    const bool is_def = first;
                    first = false;
                    const int t[4] = {L, L > 0 ? ni : 0, fb, bb};
                    tune_apply(p, t);
                    if ((st = run()) != SLOS_OK) goto done;  // warm-up
                    cudaEventRecord(e0, s);
                    for (int r = 0; r < kTuneReps && st == SLOS_OK; ++r) st = run();
                    if (st != SLOS_OK) goto done;
                    cudaEventRecord(e1, s);
                    if (cudaEventSynchronize(e1) != cudaSuccess) {
                        st = fail(SLOS_ERR_CUDA, "slos_autotune: synchronisation failed");
                        goto done;
                    }
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    ms /= kTuneReps;
                    if (is_def || ms < best * 0.995f) {
                        best = ms;
                        memcpy(best_t, t, sizeof(t));
                    }
                }
            }
        }
    }
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    tune_apply(p, best_t);
    if (st != SLOS_OK) return st;
    if (cache_path) {
        std::ofstream f(cache_path, std::ios::app);
        if (f)
            f << "{\"key\": \"" << key << "\", \"prefix_layers\": " << best_t[0] << ", \"prefix_ni\": " << best_t[1]
              << ", \"fwd_blocks_per_sm\": " << best_t[2] << ", \"bwd_blocks_per_sm\": " << best_t[3]
              << ", \"ms\": " << best << "}\n";
    }
    return SLOS_OK;
}

slos_status_t slos_plan_tuning(slos_plan_t p, int *prefix_layers_out, int *prefix_ni, int *fwd_blocks_per_sm,
                               int *bwd_blocks_per_sm) {
    if (!p || p->kind != 0) return fail(SLOS_ERR_INVALID_ARG, "slos_plan_tuning: not a single-shape plan");
    if (prefix_layers_out) *prefix_layers_out = prefix_layers(p);
    if (prefix_ni) *prefix_ni = p->tune_prefix_ni;
    if (fwd_blocks_per_sm) *fwd_blocks_per_sm = p->tune_fwd_bps;
    if (bwd_blocks_per_sm) *bwd_blocks_per_sm = p->tune_bwd_bps;
    return SLOS_OK;
}

slos_status_t slos_sync_status(slos_plan_t p, void *stream) {
    if (!p) return fail(SLOS_ERR_INVALID_ARG, "slos_sync_status: NULL plan");
    int h[16];
    cudaStream_t s = (cudaStream_t)stream;
    SLOS_CUDA(cudaMemcpyAsync(h, p->d_status, sizeof(h), cudaMemcpyDeviceToHost, s));
    SLOS_CUDA(cudaStreamSynchronize(s));
    SLOS_CUDA(cudaMemsetAsync(p->d_status, 0, 64, s));
    SLOS_CUDA(cudaStreamSynchronize(s));
    if (h[0] == SLOS_ERR_TIMEOUT)
        return fail(SLOS_ERR_TIMEOUT, "a bounded wait between layers ran out (work item " + std::to_string(h[1]) + ")");
    if (h[2] != 0)
        return fail(SLOS_ERR_TIMEOUT, "a tensor-core GEMM wait ran out (role " + std::to_string(h[2]) + ")");
    if (h[0] == kStatusBounds)
        return fail(SLOS_ERR_INTERNAL, "a device bounds check failed: index " + std::to_string(h[1]) +
                                           " past its layer (SLOS_DEBUG build)");
    if (h[0] != 0) return fail(SLOS_ERR_INTERNAL, "device status " + std::to_string(h[0]));
    return SLOS_OK;
}

slos_status_t slos_plan_destroy(slos_plan_t p) {
    if (!p) return SLOS_OK;
    if (p->d_status) cudaFree(p->d_status);
    free_tables(p);
    if (p->batched) batched_destroy(p);
    delete p;
    return SLOS_OK;
}

int64_t slos_host_rank(int m, const int *t) {
    if (!t || m < 1 || m > kMaxModes) return -1;
    return host_rank(m, t);
}

slos_status_t slos_host_unrank(int m, int k, int64_t rank, int *t) {
    if (!t || m < 1 || m > kMaxModes || k < 0 || k > 40) return fail(SLOS_ERR_INVALID_ARG, "slos_host_unrank: bad argument");
    if (rank < 0 || rank >= binom_host(m + k - 1, k)) return fail(SLOS_ERR_INVALID_ARG, "slos_host_unrank: rank out of range");
    if (m == 1) {
        t[0] = k;
        return SLOS_OK;
    }
    host_unrank(m, k, rank, t);
    return SLOS_OK;
}

slos_status_t slos_host_transition_table(int m, int k, int32_t *rowptr, uint32_t *entries, int32_t *ctab) {
    if (m < 2 || m > kMaxModes || k < 1 || k > kMaxPhotons)
        return fail(SLOS_ERR_UNSUPPORTED, "slos_host_transition_table: m in [2,24], k in [1,12]");
    if (binom_host(m + k - 2, k - 1) >= kMaxTableParent)
        return fail(SLOS_ERR_UNSUPPORTED, "slos_host_transition_table: parent layer too large for packed entries");
    std::vector<int32_t> rp, ct;
    std::vector<uint32_t> en;
    build_layer_host(m, k, rp, en, ct);
    if (rowptr) memcpy(rowptr, rp.data(), rp.size() * 4);
    if (entries) memcpy(entries, en.data(), en.size() * 4);
    if (ctab) memcpy(ctab, ct.data(), ct.size() * 4);
    return SLOS_OK;
}

slos_status_t slos_host_split_layer(int m, int n, int k, int *h, int64_t *counts, int32_t *bdesc, int32_t *bhead,
                                    int32_t *bchunk) {
    int hh = 0;
    if (m < 2 || m > kMaxModes || n < 2 || n > kMaxPhotons || k < 2 || k > n || !split_eligible(m, n, &hh))
        return fail(SLOS_ERR_UNSUPPORTED, "slos_host_split_layer: no split tables for this shape");
    SplitLayerHost L;
    split_build_layer_host(m, hh, k, L);
    if (h) *h = hh;
    if (counts) {
        counts[0] = (int64_t)L.bdesc.size() / 4;
        counts[1] = (int64_t)L.bchunk.size();
    }
    if (bdesc) memcpy(bdesc, L.bdesc.data(), L.bdesc.size() * 4);
    if (bhead) memcpy(bhead, L.bhead.data(), L.bhead.size() * 4);
    if (bchunk) memcpy(bchunk, L.bchunk.data(), L.bchunk.size() * 4);
    return SLOS_OK;
}

slos_status_t slos_host_split_tail(int m, int n, int *h, int32_t *offsets, int64_t *count, uint16_t *ctab) {
    int hh = 0;
    if (m < 2 || m > kMaxModes || n < 2 || n > kMaxPhotons || !split_eligible(m, n, &hh))
        return fail(SLOS_ERR_UNSUPPORTED, "slos_host_split_tail: no split tables for this shape");
    SplitTailHost T;
    split_build_tail_host(m, hh, n, T);
    if (h) *h = hh;
    if (offsets)
        for (int r = 0; r <= n; ++r) offsets[r] = T.coff[r];
    if (count) *count = (int64_t)T.ctab.size();
    if (ctab) memcpy(ctab, T.ctab.data(), T.ctab.size() * 2);
    return SLOS_OK;
}

slos_status_t slos_host_validate_tables(int m, int k, int kw, const uint32_t *slots, const int32_t *ctab) {
    if (m < 2 || m > kMaxModes || k < 1 || k > kMaxPhotons || (kw != 4 && kw != 8 && kw != 12) || !slots || !ctab)
        return fail(SLOS_ERR_INVALID_ARG, "slos_host_validate_tables: bad argument");
    std::string why;
    if (!tables_in_range(m, binom_host(m + k - 2, k - 1), binom_host(m + k - 1, k), kw, slots, ctab, false, &why))
        return fail(SLOS_ERR_INTERNAL, "slos_host_validate_tables: " + why);
    return SLOS_OK;
}

slos_status_t slos_inject_fault(slos_inject_t kind, int value) {
    switch (kind) {
        case SLOS_INJECT_NONE:
            g_inject_alloc.store(0);
            g_inject_stream_dev.store(-1);
            g_inject_table_budget.store(0);
            return SLOS_OK;
        case SLOS_INJECT_ALLOC_FAIL: g_inject_alloc.store(value > 0 ? value : 0); return SLOS_OK;
        case SLOS_INJECT_STREAM_DEVICE: g_inject_stream_dev.store(value >= 0 ? value : -1); return SLOS_OK;
        case SLOS_INJECT_TABLE_BUDGET: g_inject_table_budget.store(value != 0 ? 1 : 0); return SLOS_OK;
        default: return fail(SLOS_ERR_INVALID_ARG, "slos_inject_fault: unknown kind");
    }
}

slos_status_t slos_device_index_table(int m, int k, int64_t first, int64_t count, uint8_t *compositions,
                                      int32_t *parents, void *stream) {
    if (m < 2 || m > kMaxModes || k < 1 || k > kMaxPhotons)
        return fail(SLOS_ERR_UNSUPPORTED, "slos_device_index_table: m in [2,24], k in [1,12]");
    const int64_t F = binom_host(m + k - 1, k);
    if (first < 0 || count < 0 || first + count > F) return fail(SLOS_ERR_INVALID_ARG, "slos_device_index_table: range");
    if (count == 0) return SLOS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned blocks = (unsigned)((count + 127) / 128);
    ProfScope ps("slos_index_table", 0.0, s);
    switch (mmax_for(m)) {
        case 8: index_table_kernel<8><<<blocks, 128, 0, s>>>(m, k, first, count, compositions, parents); break;
        case 12: index_table_kernel<12><<<blocks, 128, 0, s>>>(m, k, first, count, compositions, parents); break;
        case 16: index_table_kernel<16><<<blocks, 128, 0, s>>>(m, k, first, count, compositions, parents); break;
        case 20: index_table_kernel<20><<<blocks, 128, 0, s>>>(m, k, first, count, compositions, parents); break;
        default: index_table_kernel<24><<<blocks, 128, 0, s>>>(m, k, first, count, compositions, parents); break;
    }
    SLOS_CUDA(cudaGetLastError());
    return SLOS_OK;
}

}  // extern "C"
