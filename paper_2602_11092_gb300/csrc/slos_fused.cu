// Whole-plan forward on chip (inference): one CTA runs every photon-number
// layer of NI instances in shared memory (Sec. II-A.2/II-A.3), so only U is
// read and only the output is written to HBM.
//
// Used for PNR table plans without activation saving whose two largest
// intermediate layers fit in shared memory for at least one instance (for
// example m=12, n=6: 4368 + 1365 states, 46 KB per instance).  Layer k lives
// in buffer (k & 1).  The U columns of all n photons are staged once, with a
// zero row (mode kMaxModes) that the padding slots name.  Two walks of the
// layers:
//
// * Fock order (slos_fwd_fused_kernel, small plans): lane = state, each state
//   reads its fixed-width parent slots once and forms the sums of all NI
//   instances (buffers complex64 [NI][cap]); output writes are coalesced.
//   Padding slots differ from lane to lane, so for plans with 8- or 12-slot
//   rows they are predicated off (a predicated-off lane sends no
//   shared-memory request, and the shared-memory pipe limits this walk).
// * Sorted order (slos_fwd_fused_sorted_kernel, plans that need 1024-thread
//   CTAs): the states of a layer sorted by their number q of occupied modes,
//   runs of equal q padded to 32 (tables.h, FusedLayer).  A warp takes a
//   block of 32 positions whose states all have q parents: one loop of q
//   slots, no padding slots, no predicates, slot rows read slot-major
//   (coalesced).  The final layer is sorted within tiles of consecutive
//   output indices and writes each output to its Fock index.  Buffers and
//   staged U hold the NI instances of an entry side by side (complex64
//   [cap][NI], swizzled in 16-byte halves), so a slot costs two vector loads
//   for all NI instances.  Measured per 4096 instances, m=12, n=6: 0.275 ms
//   in Fock order, 0.247 ms sorted with complex64 [NI][cap] buffers, 0.242 ms
//   with output tiles, 0.230 ms interleaved (0.297 ms interleaved without the
//   swizzle: bank conflicts).  The small plans are slower sorted (m=10, n=5
//   0.043 -> 0.045 ms, m=8, n=4 0.013 -> 0.017 ms: padding runs to 32 and
//   scattered writes cost more than the shorter walk saves).
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "fused.h"
#include "slos_kernels.cuh"
#include "tab_launch.h"

namespace slos {

constexpr int kFusedMaxNI = 4;
constexpr int kUsRow = kMaxModes + 1;

template <int EPI, int KW, int THREADS, bool PRED>
__device__ __forceinline__ void fused_layer(const FusedArgs &a, int k, const float2 *us, const float2 *prev,
                                            int cap_prev, float2 *cur, int cap_cur, int inst0, int ni) {
    const int Fk = a.F[k];
    const uint4 *sl = reinterpret_cast<const uint4 *>(a.slots[k]);
    const bool first = k == 1, final_layer = k == a.n;
    const size_t us_inst = (size_t)a.n * kUsRow;  // U rows of one instance
    const float2 *uk = us + (size_t)(k - 1) * kUsRow;
    for (int c = threadIdx.x; c < Fk; c += THREADS) {
        uint32_t e[KW];
#pragma unroll
        for (int q4 = 0; q4 < KW / 4; ++q4) {
            const uint4 w4 = __ldg(sl + (size_t)c * (KW / 4) + q4);
            e[4 * q4] = w4.x;
            e[4 * q4 + 1] = w4.y;
            e[4 * q4 + 2] = w4.z;
            e[4 * q4 + 3] = w4.w;
        }
        float wc = 0.f;
        if (final_layer) wc = __ldg(a.w + c);
#pragma unroll
        for (int i = 0; i < kFusedMaxNI; ++i) {
            if (i < ni) {
                const float2 *u = uk + i * us_inst;
                float2 acc;
                if (first) {
                    acc = u[e[0] & 31u];  // one photon: a_1(e_j) = U[j, c_1]
                } else {
                    const float2 *pv = prev + (size_t)i * cap_prev;
                    acc = make_float2(0.f, 0.f);
#pragma unroll
                    for (int q = 0; q < KW; ++q)
                        if (!PRED || KW == 4 || q == 0 || e[q] != kSlotEmpty)
                            acc = cfma(u[e[q] & 31u], pv[e[q] >> 5], acc);
                }
                if (!final_layer) {
                    cur[(size_t)i * cap_cur + c] = acc;
                } else if (EPI == EPI_PROBS) {
                    reinterpret_cast<float *>(a.out)[(size_t)(inst0 + i) * a.K + c] =
                        wc * (acc.x * acc.x + acc.y * acc.y);
                } else {
                    reinterpret_cast<float2 *>(a.out)[(size_t)(inst0 + i) * a.K + c] = cscale(acc, sqrtf(wc));
                }
            }
        }
    }
}

template <int EPI, int THREADS, bool PRED>
__global__ void __launch_bounds__(THREADS) slos_fwd_fused_kernel(FusedArgs a) {
    extern __shared__ float2 sm[];
    const int NI = a.NI;
    float2 *us = sm;                                  // [NI][n][kUsRow]
    float2 *buf0 = us + (size_t)NI * a.n * kUsRow;    // [NI][cap0]
    float2 *buf1 = buf0 + (size_t)NI * a.cap[0];      // [NI][cap1]
    const int inst0 = blockIdx.x * NI;
    const int ni = min(NI, a.B - inst0);
    const int nus = NI * a.n * kUsRow;
    for (int idx = threadIdx.x; idx < nus; idx += THREADS) {
        const int j = idx % kUsRow;
        const int r = idx / kUsRow;
        const int k = r % a.n, i = r / a.n;
        float2 v = make_float2(0.f, 0.f);
        if (i < ni && j < a.m) v = a.U[((size_t)(inst0 + i) * a.m + j) * a.m + a.cols[k]];
        us[idx] = v;
    }
    __syncthreads();
    for (int k = 1; k <= a.n; ++k) {
        const float2 *prev = ((k - 1) & 1) ? buf1 : buf0;
        float2 *cur = (k & 1) ? buf1 : buf0;
        const int cap_prev = a.cap[(k - 1) & 1], cap_cur = a.cap[k & 1];
        switch (a.kw[k]) {
            case 4: fused_layer<EPI, 4, THREADS, PRED>(a, k, us, prev, cap_prev, cur, cap_cur, inst0, ni); break;
            case 8: fused_layer<EPI, 8, THREADS, PRED>(a, k, us, prev, cap_prev, cur, cap_cur, inst0, ni); break;
            default: fused_layer<EPI, 12, THREADS, PRED>(a, k, us, prev, cap_prev, cur, cap_cur, inst0, ni); break;
        }
        __syncthreads();
    }
}

// The NI complex64 values (one per instance) of entry x of an array in
// shared memory: one 8-byte access, or 16-byte ones.  With NI = 4 an entry is
// two 16-byte halves whose order is swapped when bit 2 of x is set, so that
// 8 lanes reading one half of 8 random entries spread over all 8 bank
// groups (unswizzled, the first halves would sit in only 4).
template <int NI>
__device__ __forceinline__ void ld_inst(const float2 *base, uint32_t x, float2 (&v)[NI]) {
    if constexpr (NI == 1) {
        v[0] = base[x];
    } else if constexpr (NI == 2) {
        const float4 a = reinterpret_cast<const float4 *>(base)[x];
        v[0] = make_float2(a.x, a.y);
        v[1] = make_float2(a.z, a.w);
    } else {
        const float4 *e = reinterpret_cast<const float4 *>(base) + 2 * (size_t)x;
        const uint32_t sw = (x >> 2) & 1u;
        const float4 a = e[sw], b = e[sw ^ 1u];
        v[0] = make_float2(a.x, a.y);
        v[1] = make_float2(a.z, a.w);
        v[2] = make_float2(b.x, b.y);
        v[3] = make_float2(b.z, b.w);
    }
}

template <int NI>
__device__ __forceinline__ void st_inst(float2 *base, uint32_t x, const float2 (&v)[NI]) {
    if constexpr (NI == 1) {
        base[x] = v[0];
    } else if constexpr (NI == 2) {
        reinterpret_cast<float4 *>(base)[x] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    } else {
        float4 *e = reinterpret_cast<float4 *>(base) + 2 * (size_t)x;
        const uint32_t sw = (x >> 2) & 1u;
        e[sw] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
        e[sw ^ 1u] = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
    }
}

// One block of 32 positions of layer k, all with Q parents; lane = position.
// Shared memory holds the instances of a state (or of a U entry) side by
// side, so a slot costs two vector loads for all NI instances.
template <int EPI, int Q, int NI>
__device__ __forceinline__ void fused_block(const FusedArgs &a, int k, const float2 *uk, const float2 *prev,
                                            float2 *cur, int inst0, int ni, const uint32_t *row, int p) {
    const int lane = threadIdx.x & 31;
    uint32_t e[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) e[q] = __ldg(row + q * 32 + lane);
    const bool final_layer = k == a.n;
    int oc = -1;
    float wc = 0.f;
    if (final_layer) {
        oc = __ldg(a.id + p);
        wc = __ldg(a.ws + p);
    }
    float2 acc[NI];
    if (k == 1) {
        ld_inst<NI>(uk, e[0] & 31u, acc);  // one photon: a_1(e_j) = U[j, c_1]
    } else {
#pragma unroll
        for (int i = 0; i < NI; ++i) acc[i] = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            float2 u[NI], v[NI];
            ld_inst<NI>(uk, e[q] & 31u, u);
            ld_inst<NI>(prev, e[q] >> 5, v);
#pragma unroll
            for (int i = 0; i < NI; ++i) acc[i] = cfma(u[i], v[i], acc[i]);
        }
    }
    if (!final_layer) {
        st_inst<NI>(cur, (uint32_t)p, acc);
        return;
    }
    if (oc < 0) return;
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        if (i < ni) {
            if (EPI == EPI_PROBS)
                reinterpret_cast<float *>(a.out)[(size_t)(inst0 + i) * a.K + oc] =
                    wc * (acc[i].x * acc[i].x + acc[i].y * acc[i].y);
            else
                reinterpret_cast<float2 *>(a.out)[(size_t)(inst0 + i) * a.K + oc] = cscale(acc[i], sqrtf(wc));
        }
    }
}

template <int EPI, int NI>
__global__ void __launch_bounds__(1024) slos_fwd_fused_sorted_kernel(FusedArgs a) {
    extern __shared__ float2 sm[];
    float2 *us = sm;                                // [n][kUsRow][NI]
    float2 *buf0 = us + (size_t)a.n * kUsRow * NI;  // [cap0][NI]
    float2 *buf1 = buf0 + (size_t)a.cap[0] * NI;    // [cap1][NI]
    const int inst0 = blockIdx.x * NI;
    const int ni = min(NI, a.B - inst0);
    for (int r = threadIdx.x; r < a.n * kUsRow; r += 1024) {
        const int j = r % kUsRow, k = r / kUsRow;
        float2 v[NI];
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            v[i] = make_float2(0.f, 0.f);
            if (i < ni && j < a.m) v[i] = a.U[((size_t)(inst0 + i) * a.m + j) * a.m + a.cols[k]];
        }
        st_inst<NI>(us + (size_t)k * kUsRow * NI, (uint32_t)j, v);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = 1; k <= a.n; ++k) {
        const float2 *prev = ((k - 1) & 1) ? buf1 : buf0;
        float2 *cur = (k & 1) ? buf1 : buf0;
        const float2 *uk = us + (size_t)(k - 1) * kUsRow * NI;
        for (int b = warp; b < a.nblk[k]; b += 32) {
            const uint32_t info = __ldg(a.blk[k] + b);
            const uint32_t *row = a.rows[k] + (info >> 4);
            const int p = b * 32 + lane;
#define SLOS_FUSED_Q(Q) \
    case Q: fused_block<EPI, Q, NI>(a, k, uk, prev, cur, inst0, ni, row, p); break;
            switch (info & 15u) {
                SLOS_FUSED_Q(1)
                SLOS_FUSED_Q(2)
                SLOS_FUSED_Q(3)
                SLOS_FUSED_Q(4)
                SLOS_FUSED_Q(5)
                SLOS_FUSED_Q(6)
                SLOS_FUSED_Q(7)
                SLOS_FUSED_Q(8)
                SLOS_FUSED_Q(9)
                SLOS_FUSED_Q(10)
                SLOS_FUSED_Q(11)
                default: fused_block<EPI, 12, NI>(a, k, uk, prev, cur, inst0, ni, row, p); break;
            }
#undef SLOS_FUSED_Q
        }
        __syncthreads();
    }
}

size_t slos_fused_smem(int NI, int n, const int cap[2]) {
    return sizeof(float2) * ((size_t)NI * n * kUsRow + (size_t)NI * (cap[0] + cap[1]));
}

int slos_fused_max_ni() { return kFusedMaxNI; }

template <int THREADS, bool PRED>
static cudaError_t fused_attrs() {
    cudaError_t e = cudaFuncSetAttribute(slos_fwd_fused_kernel<EPI_PROBS, THREADS, PRED>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmemLimit);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(slos_fwd_fused_kernel<EPI_AMPS, THREADS, PRED>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmemLimit);
}

template <int NI>
static cudaError_t sorted_attrs() {
    cudaError_t e = cudaFuncSetAttribute(slos_fwd_fused_sorted_kernel<EPI_PROBS, NI>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmemLimit);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(slos_fwd_fused_sorted_kernel<EPI_AMPS, NI>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmemLimit);
}

template <int NI>
static cudaError_t launch_sorted(const FusedArgs &a, int epi, cudaStream_t s) {
    const unsigned grid = (unsigned)((a.B + NI - 1) / NI);
    const size_t sm = slos_fused_smem(NI, a.n, a.cap);
    if (epi == EPI_PROBS) slos_fwd_fused_sorted_kernel<EPI_PROBS, NI><<<grid, 1024, sm, s>>>(a);
    else if (epi == EPI_AMPS) slos_fwd_fused_sorted_kernel<EPI_AMPS, NI><<<grid, 1024, sm, s>>>(a);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t slos_fused_init() {
    cudaError_t e;
    if ((e = fused_attrs<512, false>()) != cudaSuccess) return e;
    if ((e = fused_attrs<512, true>()) != cudaSuccess) return e;
    if ((e = fused_attrs<1024, false>()) != cudaSuccess) return e;
    if ((e = fused_attrs<1024, true>()) != cudaSuccess) return e;
    if ((e = sorted_attrs<1>()) != cudaSuccess) return e;
    if ((e = sorted_attrs<2>()) != cudaSuccess) return e;
    return sorted_attrs<4>();
}

template <int THREADS, bool PRED>
static cudaError_t launch_fused(const FusedArgs &a, int epi, cudaStream_t s) {
    const unsigned grid = (unsigned)((a.B + a.NI - 1) / a.NI);
    const size_t sm = slos_fused_smem(a.NI, a.n, a.cap);
    if (epi == EPI_PROBS) slos_fwd_fused_kernel<EPI_PROBS, THREADS, PRED><<<grid, THREADS, sm, s>>>(a);
    else if (epi == EPI_AMPS) slos_fwd_fused_kernel<EPI_AMPS, THREADS, PRED><<<grid, THREADS, sm, s>>>(a);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template <int THREADS>
static cudaError_t launch_fused_t(const FusedArgs &a, int epi, cudaStream_t s) {
    // the predicated walk only where some layer has rows wider than 4 slots
    bool wide = false;
    for (int k = 1; k <= a.n; ++k) wide = wide || a.kw[k] > 4;
    return wide ? launch_fused<THREADS, true>(a, epi, s) : launch_fused<THREADS, false>(a, epi, s);
}

cudaError_t slos_launch_fused(const FusedArgs &a, int epi, cudaStream_t s) {
    if (a.sorted) {
        if (a.threads != 1024) return cudaErrorInvalidValue;
        switch (a.NI) {
            case 1: return launch_sorted<1>(a, epi, s);
            case 2: return launch_sorted<2>(a, epi, s);
            case 4: return launch_sorted<4>(a, epi, s);
            default: return cudaErrorInvalidValue;
        }
    }
    if (a.threads == 1024) return launch_fused_t<1024>(a, epi, s);
    if (a.threads == 512) return launch_fused_t<512>(a, epi, s);
    return cudaErrorInvalidValue;
}

}  // namespace slos
