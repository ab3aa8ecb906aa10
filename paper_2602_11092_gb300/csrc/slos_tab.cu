// Forward photon-number layer driven by the plan's transition graph
// (Sec. II-A.3): a_k(t) = sum over the entries of t of U[j, c_k] a_{k-1}(parent).
//
// Each warp owns one group of 32 instances (lane = instance) and walks a
// chunk of 32 consecutive child states.  The chunk's entries form one
// contiguous range of the CSR array: the warp loads them 32 at a time
// (coalesced), broadcasts them with shuffles, and issues 8 independent
// coalesced 256-byte parent loads per step.  U[j, c_k] for the 32 instances
// sits in shared memory (one row per mode), so the mode of an entry selects a
// row without any register indexing.  The entry's `last` bit closes a child:
// its amplitude is stored (intermediate layers) or turned into the output in
// the fused epilogue (final layer).
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "slos_kernels.cuh"
#include "tab_launch.h"

namespace slos {

template <int EPI, bool SAVE>
__global__ void __launch_bounds__(kThreads) slos_fwd_tab_kernel(FwdArgs a, TabArgs t) {
    __shared__ float2 us[kMaxModes][32];
    extern __shared__ float4 smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int grp = blockIdx.y;
    const int inst = grp * kLanes + lane;
    const bool valid = inst < a.B;
    for (int j = warp; j < a.m; j += kWarpsPerBlock)
        us[j][lane] = valid ? a.U[((int64_t)inst * a.m + j) * a.m + a.col] : make_float2(0.f, 0.f);
    __syncthreads();

    const char *prevb = reinterpret_cast<const char *>(a.prev + (int64_t)grp * a.Fprev * kLanes + lane);
    float2 *nextg = a.next + (int64_t)grp * a.Fk * kLanes + lane;
    const char *usb = reinterpret_cast<const char *>(&us[0][lane]);
    float *tile = reinterpret_cast<float *>(smem_raw) + warp * (32 * 33 * (EPI == EPI_AMPS ? 2 : 1));
    const int64_t nchunks = (a.Fk + 31) / 32;
    const int64_t wstride = (int64_t)gridDim.x * kWarpsPerBlock;
    const bool first_layer = a.k == 1;

    for (int64_t ch = (int64_t)blockIdx.x * kWarpsPerBlock + warp; ch < nchunks; ch += wstride) {
        const int64_t c0 = ch * 32;
        const int nc = (int)min((int64_t)32, a.Fk - c0);
        const int e0 = __ldg(t.rowptr + c0);
        const int e1 = __ldg(t.rowptr + c0 + nc);
        // per-child epilogue data of this chunk, one child per lane
        float wl = 0.f;
        int patl = 0;
        if (EPI != EPI_STORE && lane < nc) {
            wl = __ldg(t.w + c0 + lane);
            if (EPI == EPI_THRESH) patl = __ldg(t.pat + c0 + lane);
        }
        int ci = 0;  // child index within the chunk
        float2 acc = make_float2(0.f, 0.f);
        int run_pat = -1;
        float run_val = 0.f;
        for (int qb = e0; qb < e1; qb += 32) {
            const int cnt = min(32, e1 - qb);
            // entries past this chunk read as 0: no load, no contribution, no `last` bit
            // (a real entry is never 0: the only entry with parent 0 and mode 0 is
            // the single, hence last, entry of state (k, 0, ..., 0))
            const uint32_t mine = lane < cnt ? __ldg(t.entries + qb + lane) : 0u;
            const int nb = (cnt + 7) >> 3;
            for (int r0 = 0; r0 < 8 * nb; r0 += 8) {
                uint32_t e[8];
                float2 v[8];
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    e[r] = __shfl_sync(0xffffffffu, mine, r0 + r);
                    v[r] = make_float2(0.f, 0.f);
                    if (e[r] != 0u) {
                        v[r] = first_layer ? make_float2(1.f, 0.f)
                                           : __ldg(reinterpret_cast<const float2 *>(prevb + ((size_t)(e[r] >> 6) << 8)));
                    }
                }
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const float2 uu = *reinterpret_cast<const float2 *>(usb + (((e[r] >> 1) & 31u) << 8));
                    acc = cfma(uu, v[r], acc);
                    if (e[r] & 1u) {
                        // child c0 + ci is complete
                        const int64_t c = c0 + ci;
                        if (SAVE || EPI == EPI_STORE) nextg[c * kLanes] = acc;
                        if (EPI != EPI_STORE) {
                            const float w = __shfl_sync(0xffffffffu, wl, ci);
                            if (EPI == EPI_PROBS) {
                                tile[lane * 33 + ci] = w * (acc.x * acc.x + acc.y * acc.y);
                            } else if (EPI == EPI_AMPS) {
                                reinterpret_cast<float2 *>(tile)[lane * 33 + ci] = cscale(acc, sqrtf(w));
                            } else {
                                const float pr = w * (acc.x * acc.x + acc.y * acc.y);
                                const int pat = __shfl_sync(0xffffffffu, patl, ci);
                                if (pat != run_pat) {
                                    if (run_pat >= 0 && valid)
                                        atomicAdd(reinterpret_cast<float *>(a.out) + (int64_t)inst * a.K + run_pat,
                                                  run_val);
                                    run_pat = pat;
                                    run_val = 0.f;
                                }
                                run_val += pr;
                            }
                        }
                        acc = make_float2(0.f, 0.f);
                        ++ci;
                    }
                }
            }
        }
        if (EPI == EPI_THRESH) {
            if (run_pat >= 0 && valid)
                atomicAdd(reinterpret_cast<float *>(a.out) + (int64_t)inst * a.K + run_pat, run_val);
        }
        if (EPI == EPI_PROBS || EPI == EPI_AMPS) {
            __syncwarp();
            for (int i = 0; i < kLanes; ++i) {
                const int ii = grp * kLanes + i;
                if (ii < a.B && lane < nc) {
                    if (EPI == EPI_PROBS) {
                        reinterpret_cast<float *>(a.out)[(int64_t)ii * a.K + c0 + lane] = tile[i * 33 + lane];
                    } else {
                        reinterpret_cast<float2 *>(a.out)[(int64_t)ii * a.K + c0 + lane] =
                            reinterpret_cast<const float2 *>(tile)[i * 33 + lane];
                    }
                }
            }
            __syncwarp();
        }
    }
}

cudaError_t slos_tab_init() {
    const int sm = (int)fwd_smem_bytes(EPI_AMPS);
    cudaError_t e = cudaFuncSetAttribute(slos_fwd_tab_kernel<EPI_AMPS, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(slos_fwd_tab_kernel<EPI_AMPS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

cudaError_t slos_launch_fwd_tab(const FwdArgs &a, const TabArgs &t, int epi, bool save, int blocks_x, cudaStream_t s) {
    dim3 grid(blocks_x, a.NG);
    const size_t sm = fwd_smem_bytes(epi);
    switch (epi * 2 + (save ? 1 : 0)) {
        case 0:
        case 1: slos_fwd_tab_kernel<EPI_STORE, true><<<grid, kThreads, 0, s>>>(a, t); break;
        case 2: slos_fwd_tab_kernel<EPI_PROBS, false><<<grid, kThreads, sm, s>>>(a, t); break;
        case 3: slos_fwd_tab_kernel<EPI_PROBS, true><<<grid, kThreads, sm, s>>>(a, t); break;
        case 4: slos_fwd_tab_kernel<EPI_AMPS, false><<<grid, kThreads, sm, s>>>(a, t); break;
        case 5: slos_fwd_tab_kernel<EPI_AMPS, true><<<grid, kThreads, sm, s>>>(a, t); break;
        case 6: slos_fwd_tab_kernel<EPI_THRESH, false><<<grid, kThreads, 0, s>>>(a, t); break;
        case 7: slos_fwd_tab_kernel<EPI_THRESH, true><<<grid, kThreads, 0, s>>>(a, t); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace slos
