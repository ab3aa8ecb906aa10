// The first L photon-number layers of a table plan in one launch each way,
// every layer in shared memory (Sec. II-A.2/II-A.3).
//
// The small layers of a training step (m=16, n=8: 16, 136, 816 and 3876
// states) are too small to fill the GPU one launch per layer: each launch is
// a chain of dependent latencies (staging U, the work queue, the slot rows,
// the parent rows) that costs 10-16 us for a few microseconds of work.  Here
// one CTA takes NI instances of one 32-instance group through all L layers:
//
// * forward (slos_fwd_prefix_kernel): lane = state, each state reads its
//   fixed-width parent slots (padding slots name parent 0 and the zero row of
//   the staged U) and sums the NI instances from the previous layer in shared
//   memory; the layers the workspace needs (kept activations, and layer L,
//   which the next launch reads) are written in the group layout.
// * backward (slos_bwd_prefix_kernel): recomputes a_1..a_{L-1} on chip, reads
//   G_L, and walks layers L..1 on the child tables (lane = parent state):
//      G_{k-1}(t') = sum_j conj(U[j, c_k]) G_k(t' + e_j)
//      dU[j, c_k]  = sum_{t'} conj(a_{k-1}(t')) G_k(t' + e_j)
//   each dU column summed over the CTA in a fixed order and written as the
//   layer's single partial row of the lane's instance.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"
#include "prefix.h"
#include "slos_kernels.cuh"
#include "tab_launch.h"

namespace slos {

constexpr int kPfUsRow = kMaxModes + 1;  // U column of a photon plus a zero row (padding slots)

// ------------------------------------------------------------------ host sizing
static size_t prefix_us_bytes(int NI, int L) { return (size_t)NI * L * kPfUsRow * sizeof(float2); }
static void prefix_caps(int L, const int64_t *F, int64_t cap[2]) {
    cap[0] = cap[1] = 1;
    for (int k = 1; k <= L; ++k) cap[k & 1] = std::max(cap[k & 1], F[k]);
}
static int64_t prefix_asum(int L, const int64_t *F) {
    int64_t s = 0;
    for (int k = 0; k < L; ++k) s += F[k];
    return s;
}
size_t slos_prefix_fwd_smem(int NI, int L, const int64_t *F) {
    int64_t cap[2];
    prefix_caps(L, F, cap);
    return prefix_us_bytes(NI, L) + (size_t)NI * (cap[0] + cap[1]) * sizeof(float2);
}
size_t slos_prefix_bwd_smem(int NI, int L, const int64_t *F) {
    int64_t cap[2];
    prefix_caps(L, F, cap);
    return prefix_us_bytes(NI, L) + (size_t)NI * (prefix_asum(L, F) + cap[0] + cap[1]) * sizeof(float2);
}
int slos_prefix_layers(int m, int n, const int64_t *F) {
    if (m > kMaxModes) return 0;
    int best = 0;
    for (int L = 2; L <= n - 1; ++L)
        if (slos_prefix_bwd_smem(1, L, F) <= kPrefixInstBytes) best = L;
    return best;
}
int slos_prefix_ni(int m, int L, const int64_t *F, int batch, int sm_count) {
    (void)m;
    int ni = 1;
    while (ni * 2 <= kPrefixMaxNI && slos_prefix_bwd_smem(ni * 2, L, F) <= kPrefixSmemLimit &&
           (int64_t)batch / (ni * 2) >= 2 * (int64_t)sm_count)
        ni *= 2;
    return ni;
}

// ------------------------------------------------------------------ device
// U[j, c_k] of the CTA's instances for k = 1..L: us[(i * L + k - 1) * kPfUsRow + j],
// zero for j >= m (the padding row) and for instances past the batch.
__device__ __forceinline__ void prefix_stage_u(const PrefixArgs &a, float2 *us, int inst0, int ni) {
    const int n = a.NI * a.L * kPfUsRow;
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
        const int j = idx % kPfUsRow;
        const int r = idx / kPfUsRow;
        const int k = r % a.L, i = r / a.L;
        float2 v = make_float2(0.f, 0.f);
        if (i < ni && j < a.m) v = a.U[((size_t)(inst0 + i) * a.m + j) * a.m + a.cols[k]];
        us[idx] = v;
    }
}

// One forward layer k for the CTA's instances: prev / cur hold NI rows of
// capp / capc states.  Layer 1 reads the vacuum (a_1(e_j) = U[j, c_1]).
template <int KW>
__device__ __forceinline__ void prefix_layer(const PrefixArgs &a, int k, const float2 *us, const float2 *prev,
                                             int capp, float2 *cur, int capc, int ni, float2 *gout) {
    const int Fk = a.F[k];
    const uint4 *sl = reinterpret_cast<const uint4 *>(a.slots[k]);
#pragma unroll 2
    for (int c = threadIdx.x; c < Fk; c += blockDim.x) {
        uint32_t e[KW];
#pragma unroll
        for (int q4 = 0; q4 < KW / 4; ++q4) {
            const uint4 w4 = __ldg(sl + (size_t)c * (KW / 4) + q4);
            e[4 * q4] = w4.x;
            e[4 * q4 + 1] = w4.y;
            e[4 * q4 + 2] = w4.z;
            e[4 * q4 + 3] = w4.w;
        }
        for (int i = 0; i < ni; ++i) {
            const float2 *u = us + (size_t)(i * a.L + k - 1) * kPfUsRow;
            float2 acc;
            if (k == 1) {
                acc = u[e[0] & 31u];
            } else {
                const float2 *pv = prev + (size_t)i * capp;
                acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int q = 0; q < KW; ++q) acc = cfma(u[e[q] & 31u], pv[e[q] >> 5], acc);
            }
            cur[(size_t)i * capc + c] = acc;
            if (gout) gout[(size_t)c * kLanes + i] = acc;
        }
    }
}

__device__ __forceinline__ void prefix_layer_kw(const PrefixArgs &a, int k, const float2 *us, const float2 *prev,
                                                int capp, float2 *cur, int capc, int ni, float2 *gout) {
    switch (a.kw[k]) {
        case 4: prefix_layer<4>(a, k, us, prev, capp, cur, capc, ni, gout); break;
        case 8: prefix_layer<8>(a, k, us, prev, capp, cur, capc, ni, gout); break;
        default: prefix_layer<12>(a, k, us, prev, capp, cur, capc, ni, gout); break;
    }
}

__global__ void __launch_bounds__(kPrefixThreads, 2) slos_fwd_prefix_kernel(PrefixArgs a) {
    extern __shared__ float2 pf_sm[];
    const int NI = a.NI;
    float2 *us = pf_sm;
    float2 *buf[2];
    buf[0] = us + (size_t)NI * a.L * kPfUsRow;
    buf[1] = buf[0] + (size_t)NI * a.cap[0];
    const int inst0 = blockIdx.x * NI;
    const int ni = min(NI, a.B - inst0);
    const int grp = inst0 / kLanes, l0 = inst0 % kLanes;
    prefix_stage_u(a, us, inst0, ni);
    __syncthreads();
    for (int k = 1; k <= a.L; ++k) {
        float2 *gout = a.out[k] ? a.out[k] + ((size_t)grp * a.F[k]) * kLanes + l0 : nullptr;
        prefix_layer_kw(a, k, us, buf[(k - 1) & 1], a.cap[(k - 1) & 1], buf[k & 1], a.cap[k & 1], ni, gout);
        __syncthreads();
    }
}

// Fixed-order CTA sums of the m complex values of every thread: each warp
// reduces its values with shuffles, then thread j < m adds mode j over the
// warps in warp order and writes dst[j].  red: [warps][kMaxModes].
template <int MM>
__device__ __forceinline__ void prefix_cta_sum_modes(float2 (&du)[MM], int m, float2 *red, float2 *dst) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < MM; ++j) {
        if (j < m) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                du[j].x += __shfl_down_sync(0xffffffffu, du[j].x, o);
                du[j].y += __shfl_down_sync(0xffffffffu, du[j].y, o);
            }
            if (lane == 0) red[warp * kMaxModes + j] = du[j];
        }
    }
    __syncthreads();
    if ((int)threadIdx.x < m) {
        float2 t = make_float2(0.f, 0.f);
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t.x += red[w * kMaxModes + threadIdx.x].x;
            t.y += red[w * kMaxModes + threadIdx.x].y;
        }
        dst[threadIdx.x] = t;
    }
    __syncthreads();
}

// MM: a bound on m (16 or 24), the size of the per-thread dU accumulators.
template <int MM>
__global__ void __launch_bounds__(kPrefixThreads, 2) slos_bwd_prefix_kernel(PrefixArgs a) {
    extern __shared__ float2 pf_sm[];
    __shared__ float2 red[(kPrefixThreads / 32) * kMaxModes];
    const int NI = a.NI, L = a.L, m = a.m;
    float2 *us = pf_sm;                                  // [NI][L][kPfUsRow]
    float2 *as = us + (size_t)NI * L * kPfUsRow;         // [NI][asum]: a_0 .. a_{L-1}
    float2 *gbuf[2];                                     // G_k in gbuf[k & 1]: [NI][cap[k & 1]]
    gbuf[0] = as + (size_t)NI * a.asum;
    gbuf[1] = gbuf[0] + (size_t)NI * a.cap[0];
    int aoff[kMaxPhotons + 1];
    aoff[0] = 0;
    for (int k = 1; k <= L; ++k) aoff[k] = aoff[k - 1] + a.F[k - 1];
    const int inst0 = blockIdx.x * NI;
    const int ni = min(NI, a.B - inst0);
    const int grp = inst0 / kLanes, l0 = inst0 % kLanes;
    prefix_stage_u(a, us, inst0, ni);
    for (int i = threadIdx.x; i < NI; i += blockDim.x) as[(size_t)i * a.asum] = make_float2(1.f, 0.f);  // a_0
    // G_L of the CTA's instances
    {
        const float2 *gl = a.GL + ((size_t)grp * a.F[L]) * kLanes + l0;
        float2 *gd = gbuf[L & 1];
#pragma unroll 4
        for (int c = threadIdx.x; c < a.F[L]; c += blockDim.x)
            for (int i = 0; i < ni; ++i) gd[(size_t)i * a.cap[L & 1] + c] = gl[(size_t)c * kLanes + i];
    }
    __syncthreads();
    // a_1 .. a_{L-1}, recomputed
    for (int k = 1; k < L; ++k) {
        prefix_layer_kw(a, k, us, as + aoff[k - 1], a.asum, as + aoff[k], a.asum, ni, nullptr);
        __syncthreads();
    }
    for (int k = L; k >= 1; --k) {
        const int Fp = a.F[k - 1];
        const int32_t *ct = a.ctab[k];
        const float2 *gk = gbuf[k & 1];
        float2 *gp = gbuf[(k - 1) & 1];
        const int capk = a.cap[k & 1], capp = a.cap[(k - 1) & 1];
        for (int i = 0; i < ni; ++i) {
            const float2 *u = us + (size_t)(i * L + k - 1) * kPfUsRow;
            const float2 *ak = as + (size_t)i * a.asum + aoff[k - 1];
            const float2 *gi = gk + (size_t)i * capk;
            float2 du[MM];
#pragma unroll
            for (int j = 0; j < MM; ++j) du[j] = make_float2(0.f, 0.f);
            for (int t = threadIdx.x; t < Fp; t += blockDim.x) {
                const float2 av = ak[t];
                float2 gacc = make_float2(0.f, 0.f);
                // child ranks of parent t: rows of m entries, read as int4 when m % 4 == 0
                if (m % 4 == 0) {
                    const int4 *c4 = reinterpret_cast<const int4 *>(ct + (size_t)t * m);
#pragma unroll
                    for (int j4 = 0; j4 < MM / 4; ++j4) {
                        if (4 * j4 < m) {
                            const int4 v = __ldg(c4 + j4);
                            const int cx[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                            for (int i4 = 0; i4 < 4; ++i4) {
                                const int j = 4 * j4 + i4;
                                const float2 g = gi[cx[i4]];
                                gacc = cfma_conj_a(u[j], g, gacc);
                                du[j] = cfma_conj_a(av, g, du[j]);
                            }
                        }
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < MM; ++j) {
                        if (j < m) {
                            const float2 g = gi[__ldg(ct + (size_t)t * m + j)];
                            gacc = cfma_conj_a(u[j], g, gacc);
                            du[j] = cfma_conj_a(av, g, du[j]);
                        }
                    }
                }
                if (k >= 2) gp[(size_t)i * capp + t] = gacc;
            }
            prefix_cta_sum_modes(du, m, red, a.dUpart[k] + ((size_t)grp * kLanes + l0 + i) * m);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ launchers
cudaError_t slos_prefix_init() {
    cudaError_t e = cudaFuncSetAttribute(slos_fwd_prefix_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kPrefixSmemLimit);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(slos_bwd_prefix_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kPrefixSmemLimit);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(slos_bwd_prefix_kernel<kMaxModes>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kPrefixSmemLimit);
}

static size_t prefix_smem_args(const PrefixArgs &a, bool bwd) {
    return (size_t)a.NI * a.L * kPfUsRow * sizeof(float2) +
           (size_t)a.NI * ((bwd ? a.asum : 0) + a.cap[0] + a.cap[1]) * sizeof(float2);
}

cudaError_t slos_launch_prefix_fwd(const PrefixArgs &a, cudaStream_t s) {
    const size_t sm = prefix_smem_args(a, false);
    if (sm > kPrefixSmemLimit || a.NI < 1 || kLanes % a.NI != 0) return cudaErrorInvalidValue;
    slos_fwd_prefix_kernel<<<(a.B + a.NI - 1) / a.NI, kPrefixThreads, sm, s>>>(a);
    return cudaGetLastError();
}

cudaError_t slos_launch_prefix_bwd(const PrefixArgs &a, cudaStream_t s) {
    const size_t sm = prefix_smem_args(a, true);
    if (sm > kPrefixSmemLimit || a.NI < 1 || kLanes % a.NI != 0) return cudaErrorInvalidValue;
    const int grid = (a.B + a.NI - 1) / a.NI;
    if (a.m <= 16)
        slos_bwd_prefix_kernel<16><<<grid, kPrefixThreads, sm, s>>>(a);
    else
        slos_bwd_prefix_kernel<kMaxModes><<<grid, kPrefixThreads, sm, s>>>(a);
    return cudaGetLastError();
}

}  // namespace slos
