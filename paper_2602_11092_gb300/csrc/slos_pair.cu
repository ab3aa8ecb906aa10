// Forward photon-number layer, two instance groups per warp.
//
// a_k(t) = sum over the parents t - e_j of t of U[j, c_k] a_{k-1}(t - e_j)
// (Sec. II-A.2/II-A.3), on the plan's fixed-width slot table (tables.h).
//
// The slot-table walk spends most of its instructions on work shared by all
// instances of a state: loading and decoding the slots, forming addresses,
// branching.  Here a warp walks one state for 64 instances, the 32 of group g
// in lanes 0..15 and the 32 of group g + 1 in lanes 16..31, two adjacent
// instances per lane: each half-warp still gathers one coalesced 256-byte row
// per parent (16 bytes a lane), while the slot decode, the addresses and the
// padding branch are paid once for twice the instances.  The state is the
// warp's, so the padding branch stays uniform.
//
// Work order: CTA items of kPairWarps consecutive 32-state chunks of one group
// pair, taken from a queue in pair-major order, so the GPU sweeps the layer
// one pair (two at a boundary) at a time and the parent layer of the pair
// stays in L2 (loads marked evict-last, outputs evict-first) while each of its
// rows is read by its children.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "slos_kernels.cuh"
#include "tab_launch.h"

#include <algorithm>

namespace slos {

constexpr int kPairWarps = 4;  // one tensor-memory lane quarter per warp
constexpr int kPairThreads = kPairWarps * 32;
#ifndef SLOS_PAIR_MINB
#define SLOS_PAIR_MINB 8
#endif
constexpr int kPairMinBlocks = SLOS_PAIR_MINB;
// output tile of a warp: [64 instances][ts + 1] (one more column for the
// second group so the two halves write different banks)
#ifndef SLOS_PAIR_TS
#define SLOS_PAIR_TS 16
#endif
constexpr int pair_tile_states(int epi) { return epi == EPI_AMPS ? 16 : SLOS_PAIR_TS; }
// states per warp item; the chunk's slot rows are fetched once, one state per
// lane, and handed to the walk by shuffles
#ifndef SLOS_PAIR_CHUNK
#define SLOS_PAIR_CHUNK 16
#endif
constexpr int kPairChunk = SLOS_PAIR_CHUNK;
static_assert(kPairChunk == 16 || kPairChunk == 32, "chunk of 16 or 32 states");
size_t pair_smem_bytes(int epi) {
    if (epi != EPI_PROBS && epi != EPI_AMPS) return 0;
    const size_t cells = (size_t)kPairWarps * (64 * (pair_tile_states(epi) + 1) + 1);
    return cells * (epi == EPI_AMPS ? sizeof(float2) : sizeof(float));
}
// Tensor-memory columns per CTA: 4 per mode (the lane's two instances,
// re/im), modes 0..15 in 64 columns, 0..23 in 128 (at most 4 CTAs per SM).
constexpr int pair_tmem_cols(int m) { return m <= 16 ? 64 : 128; }

// Parent rows: read-only, not allocated in L1 (one in ten would hit there; the
// L1 data pipe is the busiest unit of the walk), kept in L2 by the policy.
__device__ __forceinline__ float4 ldg4_policy(const float4 *ptr, uint64_t pol) {
    float4 v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ void stg4_policy(float4 *ptr, float4 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(ptr), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void tm_ld4(uint32_t taddr, uint32_t (&r)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
}
// waits for the thread's outstanding tcgen05.ld; naming the loaded registers
// keeps every use of them after the wait
// waits again, naming one more group of 4 loaded registers (a wait covers
// every prior load, so the extra waits return at once)
__device__ __forceinline__ void tm_wait_tie4(uint32_t (&r)[4]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]));
}
template <int N>
__device__ __forceinline__ void tm_wait_ld4(uint32_t (&r)[N][4]) {
    static_assert(N == 4 || N == 5 || N == 6 || N == 7 || N == 8 || N == 12, "slot counts");

    if constexpr (N == 4 || N == 5) {
        asm volatile("tcgen05.wait::ld.sync.aligned;"
                     : "+r"(r[0][0]), "+r"(r[0][1]), "+r"(r[0][2]), "+r"(r[0][3]), "+r"(r[1][0]), "+r"(r[1][1]),
                       "+r"(r[1][2]), "+r"(r[1][3]), "+r"(r[2][0]), "+r"(r[2][1]), "+r"(r[2][2]), "+r"(r[2][3]),
                       "+r"(r[3][0]), "+r"(r[3][1]), "+r"(r[3][2]), "+r"(r[3][3]));
        if constexpr (N == 5) tm_wait_tie4(r[4]);
    } else if constexpr (N == 6 || N == 7) {
        asm volatile("tcgen05.wait::ld.sync.aligned;"
                     : "+r"(r[0][0]), "+r"(r[0][1]), "+r"(r[0][2]), "+r"(r[0][3]), "+r"(r[1][0]), "+r"(r[1][1]),
                       "+r"(r[1][2]), "+r"(r[1][3]), "+r"(r[2][0]), "+r"(r[2][1]), "+r"(r[2][2]), "+r"(r[2][3]),
                       "+r"(r[3][0]), "+r"(r[3][1]), "+r"(r[3][2]), "+r"(r[3][3]), "+r"(r[4][0]), "+r"(r[4][1]),
                       "+r"(r[4][2]), "+r"(r[4][3]), "+r"(r[5][0]), "+r"(r[5][1]), "+r"(r[5][2]), "+r"(r[5][3]));
        if constexpr (N == 7) tm_wait_tie4(r[6]);
    } else {
        // 8 or 12 slots: wait in two calls of 4 / 6 named groups (a wait covers every prior load)
        asm volatile("tcgen05.wait::ld.sync.aligned;"
                     : "+r"(r[0][0]), "+r"(r[0][1]), "+r"(r[0][2]), "+r"(r[0][3]), "+r"(r[1][0]), "+r"(r[1][1]),
                       "+r"(r[1][2]), "+r"(r[1][3]), "+r"(r[2][0]), "+r"(r[2][1]), "+r"(r[2][2]), "+r"(r[2][3]),
                       "+r"(r[3][0]), "+r"(r[3][1]), "+r"(r[3][2]), "+r"(r[3][3]));
        asm volatile("tcgen05.wait::ld.sync.aligned;"
                     : "+r"(r[4][0]), "+r"(r[4][1]), "+r"(r[4][2]), "+r"(r[4][3]), "+r"(r[5][0]), "+r"(r[5][1]),
                       "+r"(r[5][2]), "+r"(r[5][3]), "+r"(r[6][0]), "+r"(r[6][1]), "+r"(r[6][2]), "+r"(r[6][3]),
                       "+r"(r[7][0]), "+r"(r[7][1]), "+r"(r[7][2]), "+r"(r[7][3]));
        if constexpr (N == 12) {
            asm volatile("tcgen05.wait::ld.sync.aligned;"
                         : "+r"(r[8][0]), "+r"(r[8][1]), "+r"(r[8][2]), "+r"(r[8][3]), "+r"(r[9][0]), "+r"(r[9][1]),
                           "+r"(r[9][2]), "+r"(r[9][3]), "+r"(r[10][0]), "+r"(r[10][1]), "+r"(r[10][2]),
                           "+r"(r[10][3]), "+r"(r[11][0]), "+r"(r[11][1]), "+r"(r[11][2]), "+r"(r[11][3]));
        }
    }
}

// Sum over the first N slots of a state for the lane's two instances.  The
// mode of a slot is the warp's (the state is), so its U column address is
// warp-uniform; padding slots (mode 24) read no parent row and multiply 0.
template <int N, int KW>
__device__ __forceinline__ void pair_sum(const uint32_t (&e)[KW], const float4 *prevh, uint32_t tq, uint32_t cmask,
                                         uint64_t keep, uint32_t fprev, int *status, float2 &acc0, float2 &acc1) {
    float4 v[N];
    uint32_t u[N][4];
    (void)fprev;
    (void)status;
#pragma unroll
    for (int q = 0; q < N; ++q)
        v[q] = e[q] != kSlotEmpty ? ldg4_policy(prevh + (SLOS_IDX(e[q] >> 5, fprev, status) << 4), keep)
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int q = 0; q < N; ++q) tm_ld4(tq + 4u * (e[q] & cmask), u[q]);
    tm_wait_ld4<N>(u);
    acc0 = make_float2(0.f, 0.f);
    acc1 = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < N; ++q) {
        acc0 = cfma(make_float2(__uint_as_float(u[q][0]), __uint_as_float(u[q][1])), make_float2(v[q].x, v[q].y), acc0);
        acc1 = cfma(make_float2(__uint_as_float(u[q][2]), __uint_as_float(u[q][3])), make_float2(v[q].z, v[q].w), acc1);
    }
}

// Threshold: pattern P's probability for the lane's two instances (one
// plain store each: the pattern's states were all summed by this warp).
__device__ __forceinline__ void pair_thresh_store(const FwdArgs &a, bool hvalid, int ginst, int P, float q0, float q1,
                                                  uint64_t pol) {
    if (P < 0 || !hvalid) return;
    float *o = reinterpret_cast<float *>(a.out) + P;
    if (ginst < a.B) stg_policy(o + (int64_t)ginst * a.K, q0, pol);
    if (ginst + 1 < a.B) stg_policy(o + (int64_t)(ginst + 1) * a.K, q1, pol);
}

// Work order: each warp takes 32-state chunks of one group pair from a queue
// in pair-major order, so the GPU sweeps the layer about one pair at a time
// and the parent layer of the pair in flight stays in L2 (loads marked
// evict-last, outputs evict-first) while each of its rows is read by its
// children.  A warp restages its own U values when its chunk moves to another
// pair; no warp waits for another.
template <int EPI, bool SAVE, int KW, int TC>
__global__ void __launch_bounds__(kPairThreads, kPairMinBlocks) slos_fwd_pair_kernel(FwdArgs a, TabArgs t) {
    __shared__ uint32_t tmem_slot;
    extern __shared__ float4 smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int h = lane >> 4;         // which group of the pair
    const int sl = lane & 15;        // instances 2 sl, 2 sl + 1 of that group
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         static_cast<uint32_t>(__cvta_generic_to_shared(&tmem_slot))),
                     "r"(TC)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tq = tmem_slot + ((uint32_t)(warp * 32) << 16);
    const uint32_t cmask = TC == 64 ? 15u : 31u;  // mode -> column group (padding: a zeroed product)
    const uint64_t keep = l2_policy_keep();
    const uint64_t stream = l2_policy_stream();
    const uint4 *slots = reinterpret_cast<const uint4 *>(t.slots);
    constexpr int TS = pair_tile_states(EPI);
    constexpr int TW = 64 * (TS + 1) + 1;  // tile words per warp
    float *tile = reinterpret_cast<float *>(smem_raw) + warp * (TW * (EPI == EPI_AMPS ? 2 : 1));
    // items per pair: chunks of kPairChunk states, or (threshold) runs of whole patterns
    const int nchunks = EPI == EPI_THRESH ? t.nseg : (int)((a.Fk + kPairChunk - 1) / kPairChunk);
    const int npairs = (a.NG + 1) / 2;
    const int total = nchunks * npairs;
    const bool first_layer = a.k == 1;
    constexpr bool kSkip = KW == 8;
    int pair = -1;
    bool hvalid = false;  // this half's group exists
    int ginst = 0;        // first of the lane's two instances
    const float4 *prevh = nullptr;
    float4 *nexth = nullptr;

    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(t.work, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= total) break;
        const int pr = item / nchunks;
        if (pr != pair) {
            pair = pr;
            const int g = 2 * pair + h;
            hvalid = g < a.NG;
            ginst = g * kLanes + 2 * sl;
            // columns 4j..4j+3 of this lane: U[j, c_k] of its two instances (0 past the last mode / batch)
#pragma unroll
            for (int c16 = 0; c16 < TC; c16 += 16) {
                float vv[16];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int j = c16 / 4 + i;
                    float2 u0 = make_float2(0.f, 0.f), u1 = make_float2(0.f, 0.f);
                    if (hvalid && j < a.m) {
                        if (ginst < a.B) u0 = a.U[((int64_t)ginst * a.m + j) * a.m + a.col];
                        if (ginst + 1 < a.B) u1 = a.U[((int64_t)(ginst + 1) * a.m + j) * a.m + a.col];
                    }
                    vv[4 * i] = u0.x;
                    vv[4 * i + 1] = u0.y;
                    vv[4 * i + 2] = u1.x;
                    vv[4 * i + 3] = u1.y;
                }
                tm_st16(tq + c16, vv);
            }
            // a missing second group walks the first group's rows and writes nothing
            const int gl = hvalid ? g : 2 * pair;
            prevh = reinterpret_cast<const float4 *>(a.prev + (size_t)gl * (size_t)a.Fprev * kLanes) + sl;
            nexth = reinterpret_cast<float4 *>(a.next + (size_t)gl * (size_t)a.Fk * kLanes) + sl;
        }
        const int ch = item - pair * nchunks;
        int lo, hi;
        if (EPI == EPI_THRESH) {
            lo = __ldg(t.lseg + ch);
            hi = __ldg(t.lseg + ch + 1);
        } else {
            lo = ch * kPairChunk;
            hi = (int)min((int64_t)(lo + kPairChunk), a.Fk);
        }
        // threshold: the sum of the pattern being walked, for the lane's two instances
        int run_pat = -1;
        float run0 = 0.f, run1 = 0.f;
        // one chunk per item, or (threshold) the item's chunks in turn
        for (int cs = lo;;) {
            const uint32_t c0 = (uint32_t)cs;
            const int nc = min(kPairChunk, hi - cs);
            float wl = 0.f;
            int patl = 0, rkl = 0;
            // slot row of state c0 + lane (lanes < nc), handed out by shuffles below
            uint32_t sr[KW];
#pragma unroll
            for (int q = 0; q < KW; ++q) sr[q] = kSlotEmpty;
            if (lane < nc) {
#pragma unroll
                for (int q4 = 0; q4 < KW / 4; ++q4) {
                    const uint4 w4 = __ldg(slots + (c0 + lane) * (KW / 4) + q4);
                    sr[4 * q4] = w4.x;
                    sr[4 * q4 + 1] = w4.y;
                    sr[4 * q4 + 2] = w4.z;
                    sr[4 * q4 + 3] = w4.w;
                }
                if (EPI != EPI_STORE) wl = __ldg(t.w + c0 + lane);
                if (EPI == EPI_THRESH) {
                    patl = __ldg(t.lpat + c0 + lane);
                    if (SAVE) rkl = __ldg(t.lrank + c0 + lane);
                }
            }
            for (int ci = 0; ci < nc; ++ci) {
                const uint32_t c = c0 + (uint32_t)ci;
                uint32_t e[KW];
#pragma unroll
                for (int q = 0; q < KW; ++q) e[q] = __shfl_sync(0xffffffffu, sr[q], ci);
                float2 acc0, acc1;
                if (first_layer) {
                    uint32_t u[4][4];
                    tm_ld4(tq + 4u * (e[0] & cmask), u[0]);  // one photon: a_1(e_j) = U[j, c_1]
#pragma unroll
                    for (int q = 1; q < 4; ++q) u[q][0] = u[q][1] = u[q][2] = u[q][3] = 0u;
                    tm_wait_ld4<4>(u);
                    acc0 = make_float2(__uint_as_float(u[0][0]), __uint_as_float(u[0][1]));
                    acc1 = make_float2(__uint_as_float(u[0][2]), __uint_as_float(u[0][3]));
                } else if (kSkip && e[4] == kSlotEmpty) {
                    // at most 4 occupied modes
                    pair_sum<4>(e, prevh, tq, cmask, keep, (uint32_t)a.Fprev, a.status, acc0, acc1);
                } else if (kSkip && e[5] == kSlotEmpty) {
                    pair_sum<5>(e, prevh, tq, cmask, keep, (uint32_t)a.Fprev, a.status, acc0, acc1);
                } else if (kSkip && e[6] == kSlotEmpty) {
                    pair_sum<6>(e, prevh, tq, cmask, keep, (uint32_t)a.Fprev, a.status, acc0, acc1);
                } else if (kSkip && e[7] == kSlotEmpty) {
                    pair_sum<7>(e, prevh, tq, cmask, keep, (uint32_t)a.Fprev, a.status, acc0, acc1);
                } else {
                    pair_sum<KW>(e, prevh, tq, cmask, keep, (uint32_t)a.Fprev, a.status, acc0, acc1);
                }
                // a_n kept for the backward: at the state's Fock rank
                const uint32_t cr = (EPI == EPI_THRESH && SAVE) ? (uint32_t)__shfl_sync(0xffffffffu, rkl, ci) : c;
                if (hvalid) {
                    const float4 v = make_float4(acc0.x, acc0.y, acc1.x, acc1.y);
                    if (EPI == EPI_STORE) nexth[c << 4] = v;
                    else if (SAVE) stg4_policy(nexth + (cr << 4), v, stream);
                }
                if (EPI != EPI_STORE) {
                    const float w = __shfl_sync(0xffffffffu, wl, ci);
                    const int r0 = (32 * h + 2 * sl) * (TS + 1) + h;  // tile word of instance 2 sl, state 0
                    if (EPI == EPI_PROBS) {
                        tile[r0 + (ci & (TS - 1))] = w * (acc0.x * acc0.x + acc0.y * acc0.y);
                        tile[r0 + (TS + 1) + (ci & (TS - 1))] = w * (acc1.x * acc1.x + acc1.y * acc1.y);
                    } else if (EPI == EPI_AMPS) {
                        const float sw = sqrtf(w);
                        reinterpret_cast<float2 *>(tile)[r0 + (ci & (TS - 1))] = cscale(acc0, sw);
                        reinterpret_cast<float2 *>(tile)[r0 + (TS + 1) + (ci & (TS - 1))] = cscale(acc1, sw);
                    } else if (EPI == EPI_THRESH) {
                        // the item holds whole patterns: each sum is complete when the pattern changes
                        const int pat = __shfl_sync(0xffffffffu, patl, ci);
                        if (pat != run_pat) {
                            pair_thresh_store(a, hvalid, ginst, run_pat, run0, run1, stream);
                            run_pat = pat;
                            run0 = run1 = 0.f;
                        }
                        run0 += w * (acc0.x * acc0.x + acc0.y * acc0.y);
                        run1 += w * (acc1.x * acc1.x + acc1.y * acc1.y);
                    }
                }
                // a full tile (or the chunk's last states) goes out: TS consecutive
                // outputs of 32 / TS instances per pass
                if ((EPI == EPI_PROBS || EPI == EPI_AMPS) && ((ci & (TS - 1)) == TS - 1 || ci == nc - 1)) {
                    __syncwarp();
                    const int cb = ci & ~(TS - 1), cnt = ci - cb + 1;
                    if (EPI == EPI_PROBS && TS == 16 && (a.K & 1) == 0 &&
                        (reinterpret_cast<uintptr_t>(a.out) & 7) == 0) {
                        // rows of an even length: two consecutive outputs per lane
                        // (8-byte stores), 8 lanes per instance
                        const int il2 = 2 * (lane & 7);
                        for (int i = lane >> 3; i < 64; i += 4) {
                            const int b = 2 * pair * kLanes + i;
                            if (b < a.B && il2 < cnt) {
                                float *o = reinterpret_cast<float *>(a.out) + (int64_t)b * a.K + c0 + cb + il2;
                                const int wi = i * (TS + 1) + (i >> 5) + il2;
                                if (il2 + 1 < cnt)
                                    stg_policy(reinterpret_cast<float2 *>(o), make_float2(tile[wi], tile[wi + 1]),
                                               stream);
                                else
                                    stg_policy(o, tile[wi], stream);
                            }
                        }
                    } else {
                        const int il = lane & (TS - 1);
                        for (int i = lane / TS; i < 64; i += 32 / TS) {
                            const int b = 2 * pair * kLanes + i;
                            if (b < a.B && il < cnt) {
                                const int64_t o = (int64_t)b * a.K + c0 + cb + il;
                                const int wi = i * (TS + 1) + (i >> 5) + il;
                                if (EPI == EPI_PROBS)
                                    stg_policy(reinterpret_cast<float *>(a.out) + o, tile[wi], stream);
                                else
                                    stg_policy(reinterpret_cast<float2 *>(a.out) + o,
                                               reinterpret_cast<const float2 *>(tile)[wi], stream);
                            }
                        }
                    }
                    __syncwarp();
                }
            }
            cs += kPairChunk;
            if (EPI != EPI_THRESH || cs >= hi) break;
        }
        if (EPI == EPI_THRESH) pair_thresh_store(a, hvalid, ginst, run_pat, run0, run1, stream);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_slot), "r"(TC) : "memory");
    }
}

template <int KW, int TC>
static cudaError_t pair_attrs() {
    cudaError_t e;
    const int sp = (int)pair_smem_bytes(EPI_PROBS), sa = (int)pair_smem_bytes(EPI_AMPS);
    if ((e = cudaFuncSetAttribute(slos_fwd_pair_kernel<EPI_PROBS, false, KW, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, sp)))
        return e;
    if ((e = cudaFuncSetAttribute(slos_fwd_pair_kernel<EPI_PROBS, true, KW, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, sp)))
        return e;
    if ((e = cudaFuncSetAttribute(slos_fwd_pair_kernel<EPI_AMPS, false, KW, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, sa)))
        return e;
    return cudaFuncSetAttribute(slos_fwd_pair_kernel<EPI_AMPS, true, KW, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, sa);
}

cudaError_t slos_pair_init() {
    cudaError_t e;
    if ((e = pair_attrs<4, 64>()) != cudaSuccess) return e;
    if ((e = pair_attrs<8, 64>()) != cudaSuccess) return e;
    if ((e = pair_attrs<12, 64>()) != cudaSuccess) return e;
    if ((e = pair_attrs<4, 128>()) != cudaSuccess) return e;
    if ((e = pair_attrs<8, 128>()) != cudaSuccess) return e;
    return pair_attrs<12, 128>();
}

template <int KW, int TC>
static cudaError_t launch_pair(const FwdArgs &a, const TabArgs &t, int epi, bool save, int blocks, cudaStream_t s) {
    const size_t sm = pair_smem_bytes(epi);
    switch (epi * 2 + (save ? 1 : 0)) {
        case 0:
        case 1: slos_fwd_pair_kernel<EPI_STORE, true, KW, TC><<<blocks, kPairThreads, 0, s>>>(a, t); break;
        case 2: slos_fwd_pair_kernel<EPI_PROBS, false, KW, TC><<<blocks, kPairThreads, sm, s>>>(a, t); break;
        case 3: slos_fwd_pair_kernel<EPI_PROBS, true, KW, TC><<<blocks, kPairThreads, sm, s>>>(a, t); break;
        case 4: slos_fwd_pair_kernel<EPI_AMPS, false, KW, TC><<<blocks, kPairThreads, sm, s>>>(a, t); break;
        case 5: slos_fwd_pair_kernel<EPI_AMPS, true, KW, TC><<<blocks, kPairThreads, sm, s>>>(a, t); break;
        case 6: slos_fwd_pair_kernel<EPI_THRESH, false, KW, TC><<<blocks, kPairThreads, 0, s>>>(a, t); break;
        case 7: slos_fwd_pair_kernel<EPI_THRESH, true, KW, TC><<<blocks, kPairThreads, 0, s>>>(a, t); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Resident CTAs per SM: the register budget, and no more than the tensor
// memory (512 columns) holds.
int slos_pair_resident_blocks(int m) { return std::min(kPairMinBlocks, 512 / pair_tmem_cols(m)); }
int slos_pair_warps() { return kPairWarps; }
int slos_pair_chunk() { return kPairChunk; }

cudaError_t slos_launch_fwd_pair(const FwdArgs &a, const TabArgs &t, int epi, bool save, int blocks, cudaStream_t s) {
    const bool wide = pair_tmem_cols(a.m) == 128;
    switch (t.kw) {
        case 4: return wide ? launch_pair<4, 128>(a, t, epi, save, blocks, s) : launch_pair<4, 64>(a, t, epi, save, blocks, s);
        case 8: return wide ? launch_pair<8, 128>(a, t, epi, save, blocks, s) : launch_pair<8, 64>(a, t, epi, save, blocks, s);
        case 12:
            return wide ? launch_pair<12, 128>(a, t, epi, save, blocks, s) : launch_pair<12, 64>(a, t, epi, save, blocks, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace slos
