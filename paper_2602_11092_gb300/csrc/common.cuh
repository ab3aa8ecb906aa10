// Device-side helpers shared by the SLOS kernels.
//
// Fock-state indexing.  A composition t of k photons into m modes is written
// as a string of k stars and m-1 bars (t_0 stars, a bar, t_1 stars, ...).
// Let p_b be the distance of bar b (b = 0..m-2) from the END of the string
// (the last symbol has distance 0), so p_0 > p_1 > ... > p_{m-2} >= 0.
// Descending lexicographic order on t is descending lexicographic order on
// the strings, whose rank is the colex rank of the bar-position set:
//      rank(t) = sum_b C(p_b, m-1-b).
// Occupations: t_j = p_{j-1} - p_j - 1 with p_{-1} = k+m-1 and p_{m-1} = -1.
// Removing a photon from mode j lowers the distance of bars 0..j-1 by one, so
//      rank_{k-1}(t - e_j) = rank_k(t) - sum_{b<j} C(p_b - 1, m-2-b),
// and adding one (bars 0..j-1 move one further from the end) gives
//      rank_{k+1}(t + e_j) = rank_k(t) + sum_{b<j} C(p_b, m-2-b).
// These closed forms replace an explicit transition table (the "sparse
// transition graph" of Sec. II-A.3): the structure depends only on (m, k),
// never on U, and costs a few integer operations per (state, mode).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace slos {

constexpr int kMaxModes = 24;
constexpr int kMaxPhotons = 12;
constexpr int kBinomRows = 41;  // C(a, e) for a <= 40
constexpr int kBinomCols = 25;  // e <= 24
constexpr int kLanes = 32;      // instances per group (one per lane)

struct BinomTable {
    uint32_t v[kBinomRows][kBinomCols];
};

constexpr BinomTable make_binom_table() {
    BinomTable t{};
    for (int a = 0; a < kBinomRows; ++a) {
        for (int e = 0; e < kBinomCols; ++e) {
            if (e == 0) {
                t.v[a][e] = 1u;
            } else if (a == 0) {
                t.v[a][e] = 0u;
            } else {
                uint64_t s = (uint64_t)t.v[a - 1][e - 1] + (uint64_t)t.v[a - 1][e];
                t.v[a][e] = s > 0xffffffffull ? 0xffffffffu : (uint32_t)s;
            }
        }
    }
    return t;
}

struct FactTable {
    float v[kMaxPhotons + 2];
};

constexpr FactTable make_fact_table() {
    FactTable f{};
    double x = 1.0;
    f.v[0] = 1.0f;
    for (int i = 1; i < kMaxPhotons + 2; ++i) {
        x *= (double)i;
        f.v[i] = (float)x;
    }
    return f;
}

// One copy per translation unit, initialised at load time.
static __constant__ BinomTable c_binom = make_binom_table();
static __constant__ FactTable c_fact = make_fact_table();

// C(a, e) for a >= 0 (0 when e > a).
__device__ __forceinline__ uint32_t binom(int a, int e) { return c_binom.v[a][e]; }
// C(a - 1, e) with C(-1, e) = 0 for e >= 1 (a >= 0).
__device__ __forceinline__ uint32_t binom_m1(int a, int e) { return a > 0 ? c_binom.v[a - 1][e] : (e == 0 ? 1u : 0u); }

// ---------------------------------------------------------------- complex
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
    // c + a*b
    c.x = fmaf(a.x, b.x, c.x);
    c.x = fmaf(-a.y, b.y, c.x);
    c.y = fmaf(a.x, b.y, c.y);
    c.y = fmaf(a.y, b.x, c.y);
    return c;
}
__device__ __forceinline__ float2 cfma_conj_a(float2 a, float2 b, float2 c) {
    // c + conj(a)*b
    c.x = fmaf(a.x, b.x, c.x);
    c.x = fmaf(a.y, b.y, c.x);
    c.y = fmaf(a.x, b.y, c.y);
    c.y = fmaf(-a.y, b.x, c.y);
    return c;
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// ---------------------------------------------------------------- debug checks
// SLOS_DEBUG builds bounds-check the gather indices of the hot-path kernels:
// an index past its layer is recorded in the plan's status word (code
// kStatusBounds, then the index) and replaced by 0, a valid row, so the
// kernel finishes and the host reads the failure with slos_sync_status.
// Nothing traps.  Release builds compile the checks away.
constexpr int kStatusBounds = 7;
#ifdef SLOS_DEBUG
__device__ __forceinline__ uint32_t debug_index(uint32_t idx, uint32_t limit, int *status) {
    if (idx < limit) return idx;
    if (status && atomicCAS(status, 0, kStatusBounds) == 0) atomicExch(status + 1, (int)idx);
    return 0u;
}
#define SLOS_IDX(idx, limit, status) ::slos::debug_index((idx), (limit), (status))
#else
#define SLOS_IDX(idx, limit, status) (idx)
#endif

// ---------------------------------------------------------------- L2 hints
// L2 eviction-priority policies (createpolicy): parent rows are kept (each is
// read by up to m children spread over the layer), rows that are only
// written here are streamed.
__device__ __forceinline__ uint64_t l2_policy_keep() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_stream() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ float2 ldg_policy(const float2 *ptr, uint64_t pol) {
    float2 v;
    asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ void stg_policy(float2 *ptr, float2 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(ptr), "f"(v.x), "f"(v.y), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void stg_policy(float *ptr, float v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(ptr), "f"(v), "l"(pol) : "memory");
}

// ---------------------------------------------------------------- Fock index
// Bars of the composition with colex rank r (k photons, m modes, L = k+m-1
// symbols).  Greedy combinadic: the bar with e = m-1-b bars at or after it
// sits at the largest distance x with C(x, e) <= remaining rank.
template <int MMAX>
__device__ __forceinline__ void unrank_bars(int64_t r, int m, int L, int (&p)[MMAX]) {
    int x = L - 1;
#pragma unroll
    for (int b = 0; b < MMAX - 1; ++b) {
        if (b < m - 1) {
            const int e = m - 1 - b;
            while ((int64_t)binom(x, e) > r) --x;
            p[b] = x;
            r -= (int64_t)binom(x, e);
            --x;
        }
    }
}

// Next composition in descending-lex order (next colex bar set): the last bar
// that can move one step further from the end does so, and every bar after it
// is packed against the end.
template <int MMAX>
__device__ __forceinline__ void next_bars(int m, int L, int (&p)[MMAX]) {
    int bstar = -1;
#pragma unroll
    for (int b = 0; b < MMAX - 1; ++b) {
        if (b < m - 1) {
            const int prevp = (b == 0) ? L : p[b - 1];
            if (p[b] + 1 < prevp) bstar = b;
        }
    }
#pragma unroll
    for (int b = 0; b < MMAX - 1; ++b) {
        if (b < m - 1) {
            if (b == bstar) p[b] += 1;
            else if (b > bstar) p[b] = m - 2 - b;
        }
    }
}

// Occupation of mode j from the bars (j compile-time inside unrolled loops).
template <int MMAX>
__device__ __forceinline__ int occupation(int j, int m, int L, const int (&p)[MMAX]) {
    const int hi = (j == 0) ? L : p[j - 1];
    const int lo = (j < m - 1) ? p[j] : -1;
    return hi - lo - 1;
}

// Colex rank of a k-subset given as a bitmask: sum_i C(q_i, i), q_1 < q_2 < ...
__device__ __forceinline__ uint32_t colex_rank(uint32_t mask) {
    uint32_t r = 0;
    int i = 1;
    while (mask) {
        const int q = __ffs(mask) - 1;
        r += binom(q, i);
        ++i;
        mask &= mask - 1;
    }
    return r;
}


// ---------------------------------------------------------------- bar masks
// The same state as a bitmask of bar positions (bit p_b set).  Descending-lex
// order on compositions is colex order on bar sets, i.e. increasing integer
// order among masks with m-1 bits set, so the successor is the next larger
// integer with the same popcount (Gosper's next-combination step).
template <int MMAX>
struct BarMask {
    // up to 20 modes and 12 photons the string has at most 31 symbols
    using T = typename std::conditional<(MMAX + kMaxPhotons - 1 <= 32), uint32_t, unsigned long long>::type;
};

__device__ __forceinline__ uint32_t next_comb(uint32_t z) {
    const uint32_t c = z & (0u - z);
    const uint32_t r = z + c;
    return r | (((r ^ z) >> 2) >> (__ffs(z) - 1));
}
__device__ __forceinline__ unsigned long long next_comb(unsigned long long z) {
    const unsigned long long c = z & (0ull - z);
    const unsigned long long r = z + c;
    return r | (((r ^ z) >> 2) >> (__ffsll((long long)z) - 1));
}
// Highest set bit position of a nonzero mask.
__device__ __forceinline__ int top_bit(uint32_t z) { return 31 - __clz(z); }
__device__ __forceinline__ int top_bit(unsigned long long z) { return 63 - __clzll((long long)z); }

template <int MMAX, typename Z>
__device__ __forceinline__ Z unrank_mask(int64_t r, int m, int L) {
    int p[MMAX];
    unrank_bars<MMAX>(r, m, L, p);
    Z z = 0;
#pragma unroll
    for (int b = 0; b < MMAX - 1; ++b)
        if (b < m - 1) z |= (Z)1 << p[b];
    return z;
}

}  // namespace slos
