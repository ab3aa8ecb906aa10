// Forward photon-number layer driven by the plan's transition graph
// (Sec. II-A.3): a_k(t) = sum over the parents t - e_j of t of
// U[j, c_k] a_{k-1}(t - e_j).
//
// The graph of layer k is a fixed-width slot table: state c has KW slots
// (parent rank << 5 | mode j for every occupied mode, then kSlotEmpty, which
// names parent 0 and a zero row of U).  Each warp owns one group of 32
// instances (lane = instance) and walks a chunk of 32 consecutive states,
// one state per step: the state's slots arrive as 16-byte broadcast loads,
// its parent rows (coalesced 256-byte loads) are issued together, and the
// sum runs over them without per-slot branches.  The state is the same for
// the whole warp (lane = instance), so in intermediate layers a uniform
// branch on the first padding slot picks a body of 4, 6 or 8 slots for
// 8-slot rows: padding then costs no parent-row or U-row reads.  U[j, c_k]
// for the 32 instances sits in shared memory, one row per mode plus the zero
// row.  The register budget (fwd_tab_min_blocks resident blocks) keeps
// enough warps in flight to cover the latency of each warp's chain (slot
// row, gathers, sums); at 64 warps per SM the final layer is bound by the L1
// pipe.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "slos_kernels.cuh"
#include "tab_launch.h"

namespace slos {

// sum over the first N slots of a state: the N parent rows are issued
// together, then N complex multiply-adds with the staged U rows
template <int N, int KW>
__device__ __forceinline__ float2 parent_sum(const uint32_t (&e)[KW], const float2 *prevg, const float2 *usl) {
    float2 v[N];
#pragma unroll
    for (int q = 0; q < N; ++q) v[q] = __ldg(prevg + ((e[q] >> 5) << 5));
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < N; ++q) acc = cfma(usl[(e[q] & 31u) * 32u], v[q], acc);
    return acc;
}

// U[j, c_k] in tensor memory (UT kernels).  Every slot of the shared-memory
// version reads a 256-byte U row through the L1 pipe (two wavefronts, twice
// what the parent-row gather itself costs); instead each 32-lane quarter of
// the CTA's tensor memory holds the group's U values, column pair 2j, 2j+1 =
// U[j, c_k] (zero for the padding mode 24), and a state fetches one pair per
// slot with tcgen05.ld, issued together and awaited once.  The slot's mode
// is the warp's (lane = instance), so the column address is warp-uniform.
// Warps w and w + 4 share lane quarter w mod 4, which holds the same values.
constexpr int kTabTmemCols = 64;

__device__ __forceinline__ void tm_ld2(uint32_t taddr, uint32_t &r0, uint32_t &r1) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(taddr));
}
// waits for the thread's outstanding tcgen05.ld; naming the loaded registers
// keeps every use of them after the wait
template <int N>
__device__ __forceinline__ void tm_wait_ld_n(uint32_t (&r)[N][2]) {
    static_assert(N == 4 || N == 6 || N == 8 || N == 12, "slot counts");
    if constexpr (N == 4) {
        asm volatile("tcgen05.wait::ld.sync.aligned;"
                     : "+r"(r[0][0]), "+r"(r[0][1]), "+r"(r[1][0]), "+r"(r[1][1]), "+r"(r[2][0]), "+r"(r[2][1]),
                       "+r"(r[3][0]), "+r"(r[3][1]));
    } else if constexpr (N == 6) {
        asm volatile("tcgen05.wait::ld.sync.aligned;"
                     : "+r"(r[0][0]), "+r"(r[0][1]), "+r"(r[1][0]), "+r"(r[1][1]), "+r"(r[2][0]), "+r"(r[2][1]),
                       "+r"(r[3][0]), "+r"(r[3][1]), "+r"(r[4][0]), "+r"(r[4][1]), "+r"(r[5][0]), "+r"(r[5][1]));
    } else if constexpr (N == 8) {
        asm volatile("tcgen05.wait::ld.sync.aligned;"
                     : "+r"(r[0][0]), "+r"(r[0][1]), "+r"(r[1][0]), "+r"(r[1][1]), "+r"(r[2][0]), "+r"(r[2][1]),
                       "+r"(r[3][0]), "+r"(r[3][1]), "+r"(r[4][0]), "+r"(r[4][1]), "+r"(r[5][0]), "+r"(r[5][1]),
                       "+r"(r[6][0]), "+r"(r[6][1]), "+r"(r[7][0]), "+r"(r[7][1]));
    } else {
        asm volatile("tcgen05.wait::ld.sync.aligned;"
                     : "+r"(r[0][0]), "+r"(r[0][1]), "+r"(r[1][0]), "+r"(r[1][1]), "+r"(r[2][0]), "+r"(r[2][1]),
                       "+r"(r[3][0]), "+r"(r[3][1]), "+r"(r[4][0]), "+r"(r[4][1]), "+r"(r[5][0]), "+r"(r[5][1]),
                       "+r"(r[6][0]), "+r"(r[6][1]), "+r"(r[7][0]), "+r"(r[7][1]), "+r"(r[8][0]), "+r"(r[8][1]),
                       "+r"(r[9][0]), "+r"(r[9][1]), "+r"(r[10][0]), "+r"(r[10][1]), "+r"(r[11][0]),
                       "+r"(r[11][1]));
    }
}

// sum over the first N slots of a state: the N parent rows are issued
// together, then N complex multiply-adds with the staged U rows
template <int N, int KW, bool UT>
__device__ __forceinline__ float2 parent_sum_keep(const uint32_t (&e)[KW], const float2 *prevg, const float2 *usl,
                                                  uint32_t tq, uint64_t pol) {
    float2 v[N];
#pragma unroll
    for (int q = 0; q < N; ++q) v[q] = ldg_policy(prevg + ((e[q] >> 5) << 5), pol);
    float2 acc = make_float2(0.f, 0.f);
    if constexpr (UT) {
        uint32_t u[N][2];
#pragma unroll
        for (int q = 0; q < N; ++q) tm_ld2(tq + 2u * (e[q] & 31u), u[q][0], u[q][1]);
        tm_wait_ld_n<N>(u);
#pragma unroll
        for (int q = 0; q < N; ++q)
            acc = cfma(make_float2(__uint_as_float(u[q][0]), __uint_as_float(u[q][1])), v[q], acc);
    } else {
#pragma unroll
        for (int q = 0; q < N; ++q) acc = cfma(usl[(e[q] & 31u) * 32u], v[q], acc);
    }
    return acc;
}

// Work order.  Each CTA takes items of kWarpsPerBlock consecutive 32-state
// chunks of one instance group from a queue in group-major order, so the GPU
// sweeps the layer one group (two at a group boundary) at a time: the parent
// layer of one group stays in L2 (marked evict-last) while each of its rows
// is read by its m children, instead of the parent layers of all groups
// competing for L2 with the streamed outputs.  The CTA restages the U rows
// when its item moves to another group.
template <int EPI, bool SAVE, int KW, bool UT>
__global__ void __launch_bounds__(kThreads, fwd_tab_min_blocks(EPI)) slos_fwd_tab_kernel(FwdArgs a, TabArgs t) {
    __shared__ float2 us[kMaxModes + 1][32];
    __shared__ int s_item;
    __shared__ uint32_t tmem_slot;
    extern __shared__ float4 smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    if (warp == 0) us[kMaxModes][lane] = make_float2(0.f, 0.f);
    if (UT && warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         static_cast<uint32_t>(__cvta_generic_to_shared(&tmem_slot))),
                     "r"(kTabTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (UT) asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (UT) asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tq = UT ? tmem_slot + ((uint32_t)((warp & 3) * 32) << 16) : 0u;
    const uint64_t keep = l2_policy_keep();
    const uint64_t stream = l2_policy_stream();
    const float2 *usl = &us[0][lane];
    const uint4 *slots = reinterpret_cast<const uint4 *>(t.slots);
    constexpr int TS = kFwdTabTile;  // states per output tile
    float *tile = reinterpret_cast<float *>(smem_raw) + warp * (32 * (TS + 1) * (EPI == EPI_AMPS ? 2 : 1));
    const int64_t nchunks = (a.Fk + 31) / 32;
    const int total = t.items_per_group * a.NG;
    const bool first_layer = a.k == 1;
    // intermediate layers with 8-slot rows branch to a 4-, 6- or 8-slot body
    // (measured on the m=16, n=8 step: 0.404 -> 0.361 ms; the final layer
    // is slower with the branch at its 32-register budget, 0.879 -> 0.936 ms)
    constexpr bool kSkip = KW == 8 && (EPI == EPI_STORE || UT);
    int grp = -1, inst = 0;
    bool valid = false;
    const float2 *prevg = nullptr;
    float2 *nextg = nullptr;

    for (;;) {
        __syncthreads();  // the previous item's U rows and queue slot are no longer read
        if (threadIdx.x == 0) s_item = atomicAdd(t.work, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= total) break;
        const int g = item / t.items_per_group;
        if (g != grp) {
            grp = g;
            inst = grp * kLanes + lane;
            valid = inst < a.B;
            if (!UT) {
                for (int j = warp; j < a.m; j += kWarpsPerBlock)
                    us[j][lane] = valid ? a.U[((int64_t)inst * a.m + j) * a.m + a.col] : make_float2(0.f, 0.f);
            } else if (warp < 4) {
                // columns 2j, 2j+1 of this lane = U[j, c_k] of its instance (0 past the last mode)
#pragma unroll
                for (int c16 = 0; c16 < kTabTmemCols; c16 += 16) {
                    float v[16];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int j = c16 / 2 + i;
                        float2 u = make_float2(0.f, 0.f);
                        if (valid && j < a.m) u = a.U[((int64_t)inst * a.m + j) * a.m + a.col];
                        v[2 * i] = u.x;
                        v[2 * i + 1] = u.y;
                    }
                    tm_st16(tq + c16, v);
                }
            }
            // 64-bit group bases once; per-state offsets are 32-bit (table plans: F * 32 < 2^31)
            prevg = a.prev + (size_t)grp * (size_t)a.Fprev * kLanes + lane;
            nextg = a.next + (size_t)grp * (size_t)a.Fk * kLanes + lane;
            if (UT) asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            if (UT) asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
        const int64_t ch = (int64_t)(item - g * t.items_per_group) * kWarpsPerBlock + warp;
        if (ch >= nchunks) continue;
        const uint32_t c0 = (uint32_t)ch * 32u;
        const int nc = (int)min((int64_t)32, a.Fk - (int64_t)c0);
        float wl = 0.f;
        int patl = 0;
        if (EPI != EPI_STORE && lane < nc) {
            wl = __ldg(t.w + c0 + lane);
            if (EPI == EPI_THRESH) patl = __ldg(t.pat + c0 + lane);
        }
        int run_pat = -1;
        float run_val = 0.f;
        for (int ci = 0; ci < nc; ++ci) {
            const uint32_t c = c0 + (uint32_t)ci;
            uint32_t e[KW];
#pragma unroll
            for (int q4 = 0; q4 < KW / 4; ++q4) {
                const uint4 w4 = __ldg(slots + c * (KW / 4) + q4);
                e[4 * q4] = w4.x;
                e[4 * q4 + 1] = w4.y;
                e[4 * q4 + 2] = w4.z;
                e[4 * q4 + 3] = w4.w;
            }
            float2 acc;
            if (first_layer) {
                if (UT) {
                    uint32_t u[4][2] = {{0u, 0u}, {0u, 0u}, {0u, 0u}, {0u, 0u}};
                    tm_ld2(tq + 2u * (e[0] & 31u), u[0][0], u[0][1]);
                    tm_wait_ld_n<4>(u);
                    acc = make_float2(__uint_as_float(u[0][0]), __uint_as_float(u[0][1]));
                } else {
                    acc = usl[(e[0] & 31u) * 32u];  // one photon: a_1(e_j) = U[j, c_1]
                }
            } else if (kSkip && e[4] == kSlotEmpty) {
                acc = parent_sum_keep<4, KW, UT>(e, prevg, usl, tq, keep);  // at most 4 occupied modes
            } else if (kSkip && e[6] == kSlotEmpty) {
                acc = parent_sum_keep<6, KW, UT>(e, prevg, usl, tq, keep);
            } else {
                acc = parent_sum_keep<KW, KW, UT>(e, prevg, usl, tq, keep);
            }
            if (EPI == EPI_STORE) nextg[c << 5] = acc;
            else if (SAVE) stg_policy(nextg + (c << 5), acc, stream);
            if (EPI != EPI_STORE) {
                const float w = __shfl_sync(0xffffffffu, wl, ci);
                if (EPI == EPI_PROBS) {
                    tile[lane * (TS + 1) + (ci & (TS - 1))] = w * (acc.x * acc.x + acc.y * acc.y);
                } else if (EPI == EPI_AMPS) {
                    reinterpret_cast<float2 *>(tile)[lane * (TS + 1) + (ci & (TS - 1))] = cscale(acc, sqrtf(w));
                } else if (EPI == EPI_THRESH) {
                    const int pat = __shfl_sync(0xffffffffu, patl, ci);
                    const float pr = w * (acc.x * acc.x + acc.y * acc.y);
                    if (pat != run_pat) {
                        if (run_pat >= 0 && valid)
                            atomicAdd(reinterpret_cast<float *>(a.out) + (int64_t)inst * a.K + run_pat, run_val);
                        run_pat = pat;
                        run_val = 0.f;
                    }
                    run_val += pr;
                }
            }
            // a full tile (or the chunk's last states) goes out: 32 / TS
            // instances per pass, TS consecutive outputs each
            if ((EPI == EPI_PROBS || EPI == EPI_AMPS) && ((ci & (TS - 1)) == TS - 1 || ci == nc - 1)) {
                __syncwarp();
                const int cb = ci & ~(TS - 1), cnt = ci - cb + 1;
                const int il = lane & (TS - 1);
                for (int i = lane / TS; i < kLanes; i += 32 / TS) {
                    const int ii = grp * kLanes + i;
                    if (ii < a.B && il < cnt) {
                        const int64_t o = (int64_t)ii * a.K + c0 + cb + il;
                        if (EPI == EPI_PROBS) {
                            stg_policy(reinterpret_cast<float *>(a.out) + o, tile[i * (TS + 1) + il], stream);
                        } else {
                            stg_policy(reinterpret_cast<float2 *>(a.out) + o,
                                       reinterpret_cast<const float2 *>(tile)[i * (TS + 1) + il], stream);
                        }
                    }
                }
                __syncwarp();
            }
        }
        if (EPI == EPI_THRESH && run_pat >= 0 && valid)
            atomicAdd(reinterpret_cast<float *>(a.out) + (int64_t)inst * a.K + run_pat, run_val);
    }
    if (UT) {
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (warp == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_slot), "r"(kTabTmemCols)
                         : "memory");
        }
    }
}

template <int KW>
static cudaError_t tab_attrs() {
    cudaError_t e;
    const int sp = (int)fwd_tab_smem_bytes(EPI_PROBS), sa = (int)fwd_tab_smem_bytes(EPI_AMPS);
    if ((e = cudaFuncSetAttribute(slos_fwd_tab_kernel<EPI_PROBS, false, KW, kFwdTabTmemU>, cudaFuncAttributeMaxDynamicSharedMemorySize, sp)))
        return e;
    if ((e = cudaFuncSetAttribute(slos_fwd_tab_kernel<EPI_PROBS, true, KW, kFwdTabTmemU>, cudaFuncAttributeMaxDynamicSharedMemorySize, sp)))
        return e;
    if ((e = cudaFuncSetAttribute(slos_fwd_tab_kernel<EPI_AMPS, false, KW, kFwdTabTmemU>, cudaFuncAttributeMaxDynamicSharedMemorySize, sa)))
        return e;
    return cudaFuncSetAttribute(slos_fwd_tab_kernel<EPI_AMPS, true, KW, kFwdTabTmemU>, cudaFuncAttributeMaxDynamicSharedMemorySize, sa);
}

cudaError_t slos_tab_init() {
    cudaError_t e;
    if ((e = tab_attrs<4>()) != cudaSuccess) return e;
    if ((e = tab_attrs<8>()) != cudaSuccess) return e;
    return tab_attrs<12>();
}

template <int KW>
static cudaError_t launch_tab(const FwdArgs &a, const TabArgs &t, int epi, bool save, int blocks_x, cudaStream_t s) {
    const dim3 grid(blocks_x);
    const size_t sm = fwd_tab_smem_bytes(epi);
    switch (epi * 2 + (save ? 1 : 0)) {
        case 0:
        case 1: slos_fwd_tab_kernel<EPI_STORE, true, KW, kFwdTabTmemU><<<grid, kThreads, 0, s>>>(a, t); break;
        case 2: slos_fwd_tab_kernel<EPI_PROBS, false, KW, kFwdTabTmemU><<<grid, kThreads, sm, s>>>(a, t); break;
        case 3: slos_fwd_tab_kernel<EPI_PROBS, true, KW, kFwdTabTmemU><<<grid, kThreads, sm, s>>>(a, t); break;
        case 4: slos_fwd_tab_kernel<EPI_AMPS, false, KW, kFwdTabTmemU><<<grid, kThreads, sm, s>>>(a, t); break;
        case 5: slos_fwd_tab_kernel<EPI_AMPS, true, KW, kFwdTabTmemU><<<grid, kThreads, sm, s>>>(a, t); break;
        case 6: slos_fwd_tab_kernel<EPI_THRESH, false, KW, kFwdTabTmemU><<<grid, kThreads, 0, s>>>(a, t); break;
        case 7: slos_fwd_tab_kernel<EPI_THRESH, true, KW, kFwdTabTmemU><<<grid, kThreads, 0, s>>>(a, t); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t slos_launch_fwd_tab(const FwdArgs &a, const TabArgs &t, int epi, bool save, int blocks_x, cudaStream_t s) {
    switch (t.kw) {
        case 4: return launch_tab<4>(a, t, epi, save, blocks_x, s);
        case 8: return launch_tab<8>(a, t, epi, save, blocks_x, s);
        case 12: return launch_tab<12>(a, t, epi, save, blocks_x, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace slos
