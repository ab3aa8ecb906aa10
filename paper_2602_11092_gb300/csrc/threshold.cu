// Threshold detection (the detector model of Sec. 3.1: a threshold detector
// only registers whether its mode holds any photon).  The outcome with
// occupied-mode set b has probability
//      q(b) = sum of p(t) over the Fock states t of n photons with support b,
// and those states are t = 1_b + u for the compositions u of n - |b| photons
// over the |b| modes of b: C(n-1, |b|-1) of them.
//
// The final SLOS layer stores a_n ([NG][F_n][32] complex64, one 256-byte row
// per state).  This kernel then forms each q(b) of each instance as one sum
// in a fixed order (u in descending-lex order), so the outputs are the same
// bit for bit from run to run, written with plain stores and nothing to
// clear first.  Patterns are in output order: |b| = 1..min(n, m), then colex
// order of b.  A warp takes 32 consecutive patterns of one instance group.
// For each pattern its lanes rank up to 32 of the pattern's states at once
// (the Fock rank from the bar formula of common.cuh, and prod t_j!), then the
// warp reads those states' rows in order, lane = instance, and accumulates
// w_t |a_n(t)|^2.  The 32 x 32 results leave through a shared-memory tile as
// 128-byte segments of the rows of out[B][K].
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "slos_kernels.cuh"

namespace slos {

constexpr int kThreshWarps = 8;

// Pattern P of class j (|b| = j): its modes q_1 < ... < q_j, colex unranked.
__device__ __forceinline__ uint32_t pattern_mask(int64_t r, int j, int m) {
    uint32_t mask = 0;
    int x = m - 1;
    for (int i = j; i >= 1; --i) {
        while ((int64_t)binom(x, i) > r) --x;
        r -= (int64_t)binom(x, i);
        mask |= 1u << x;
        --x;
    }
    return mask;
}

// State number r (descending-lex order of u) of the pattern with support
// `mask` (j modes): its Fock rank in layer n and prod t_j!.  The bars of u (a
// composition of n - j photons over j modes, Lu = n - 1 symbols) come out of
// the greedy combinadic unranking of common.cuh's unrank_bars one by one, in
// the order the modes of the pattern consume them.
__device__ __forceinline__ void pattern_state(int64_t r, uint32_t mask, int j, int m, int n, uint32_t &rank,
                                              float &fact) {
    const int Lu = n - 1;
    int x = Lu - 1;     // next candidate bar distance of u
    int prev = Lu, i = 0;
    int p = n + m - 1;  // bar distances of t, p_{-1} = L
    rank = 0;
    fact = 1.f;
    for (int mode = 0; mode < m; ++mode) {
        int tm = 0;
        if ((mask >> mode) & 1u) {
            int lo = -1;
            if (i < j - 1) {
                const int e = j - 1 - i;
                while ((int64_t)binom(x, e) > r) --x;
                r -= (int64_t)binom(x, e);
                lo = x--;
            }
            tm = prev - lo;  // u_i + 1
            prev = lo;
            ++i;
            fact *= c_fact.v[tm];
        }
        if (mode < m - 1) {
            p -= tm + 1;
            rank += binom(p, m - 1 - mode);
        }
    }
}

__global__ void __launch_bounds__(kThreshWarps * 32) slos_thresh_sum_kernel(ThreshArgs a) {
    __shared__ float tile[kThreshWarps][32][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = blockIdx.y;
    const int64_t P0 = ((int64_t)blockIdx.x * kThreshWarps + warp) * 32;
    if (P0 >= a.K) return;
    const int np = (int)min((int64_t)32, a.K - P0);
    const float2 *ag = a.an + (size_t)g * (size_t)a.Fn * kLanes + lane;
    float(*t)[33] = tile[warp];
    for (int pi = 0; pi < np; ++pi) {
        const int64_t P = P0 + pi;
        // class j = |b|: the C(m, 1) + ... + C(m, j-1) patterns before it
        int j = 1;
        int64_t off = 0;
        while (j < a.jmax && off + (int64_t)binom(a.m, j) <= P) off += (int64_t)binom(a.m, j++);
        const uint32_t mask = pattern_mask(P - off, j, a.m);
        const int64_t nst = (int64_t)binom(a.n - 1, j - 1);
        float acc = 0.f;
        for (int64_t r0 = 0; r0 < nst; r0 += 32) {
            uint32_t rk = 0;
            float fw = 0.f;
            if (r0 + lane < nst) pattern_state(r0 + lane, mask, j, a.m, a.n, rk, fw);
            const int cnt = (int)min((int64_t)32, nst - r0);
            int i = 0;
            for (; i + 4 <= cnt; i += 4) {
                float2 v[4];
                float f[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t c = SLOS_IDX(__shfl_sync(0xffffffffu, rk, i + q), (uint32_t)a.Fn, a.status);
                    f[q] = __shfl_sync(0xffffffffu, fw, i + q);
                    v[q] = __ldcs(ag + (size_t)c * kLanes);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) acc += f[q] * (v[q].x * v[q].x + v[q].y * v[q].y);
            }
            for (; i < cnt; ++i) {
                const uint32_t c = SLOS_IDX(__shfl_sync(0xffffffffu, rk, i), (uint32_t)a.Fn, a.status);
                const float f = __shfl_sync(0xffffffffu, fw, i);
                const float2 v = __ldcs(ag + (size_t)c * kLanes);
                acc += f * (v.x * v.x + v.y * v.y);
            }
        }
        t[lane][pi] = acc * a.inv_sfact;
    }
    __syncwarp();
    for (int i = 0; i < 32; ++i) {
        const int b = g * kLanes + i;
        if (b < a.B && lane < np) a.out[(int64_t)b * a.K + P0 + lane] = t[i][lane];
    }
}

cudaError_t slos_launch_thresh_sum(const ThreshArgs &a, cudaStream_t s) {
    const int64_t blocks = (a.K + 32 * kThreshWarps - 1) / (32 * kThreshWarps);
    if (blocks > 0x7fffffff || a.NG > 65535) return cudaErrorInvalidValue;
    slos_thresh_sum_kernel<<<dim3((unsigned)blocks, a.NG), kThreshWarps * 32, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace slos
