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

template <int EPI, bool SAVE, int GPW>
__global__ void __launch_bounds__(kThreads, kFwdTabMinBlocks) slos_fwd_tab_kernel(FwdArgs a, TabArgs t) {
    // GPW groups of 32 instances per warp: lane l serves instance l of each
    // group, so the entry stream and its decoding are shared by 32*GPW instances.
    __shared__ float2 us[GPW][kMaxModes][32];
    extern __shared__ float4 smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int grp0 = blockIdx.y * GPW;
    bool valid[GPW];
    int inst[GPW];
#pragma unroll
    for (int q = 0; q < GPW; ++q) {
        inst[q] = (grp0 + q) * kLanes + lane;
        valid[q] = (grp0 + q) < a.NG && inst[q] < a.B;
    }
    for (int j = warp; j < a.m; j += kWarpsPerBlock) {
#pragma unroll
        for (int q = 0; q < GPW; ++q)
            us[q][j][lane] = valid[q] ? a.U[((int64_t)inst[q] * a.m + j) * a.m + a.col] : make_float2(0.f, 0.f);
    }
    __syncthreads();

    // 64-bit group bases once; every per-entry offset below is 32-bit
    // (table plans have F_k * 32 < 2^32)
    const float2 *prevg[GPW];
    float2 *nextg[GPW];
#pragma unroll
    for (int q = 0; q < GPW; ++q) {
        const int g = min(grp0 + q, a.NG - 1);  // a missing second group reads group NG-1 and writes nothing
        prevg[q] = a.prev + (size_t)g * (size_t)a.Fprev * kLanes + lane;
        nextg[q] = a.next + (size_t)g * (size_t)a.Fk * kLanes + lane;
    }
    const char *usb = reinterpret_cast<const char *>(&us[0][0][lane]);
    constexpr int kUsGroup = kMaxModes * 32 * 8;  // bytes between the groups' U tables
    float *tile = reinterpret_cast<float *>(smem_raw) + warp * (GPW * 32 * 33 * (EPI == EPI_AMPS ? 2 : 1));
    const int64_t nchunks = (a.Fk + 31) / 32;
    const int64_t wstride = (int64_t)gridDim.x * kWarpsPerBlock;
    const bool first_layer = a.k == 1;

    for (int64_t ch = (int64_t)blockIdx.x * kWarpsPerBlock + warp; ch < nchunks; ch += wstride) {
        const int64_t c0 = ch * 32;
        const int nc = (int)min((int64_t)32, a.Fk - c0);
        const int e0 = __ldg(t.rowptr + c0);
        const int e1 = __ldg(t.rowptr + c0 + nc);
        float wl = 0.f;
        int patl = 0;
        if (EPI != EPI_STORE && lane < nc) {
            wl = __ldg(t.w + c0 + lane);
            if (EPI == EPI_THRESH) patl = __ldg(t.pat + c0 + lane);
        }
        int ci = 0;
        float2 acc[GPW];
        int run_pat[GPW];
        float run_val[GPW];
#pragma unroll
        for (int q = 0; q < GPW; ++q) {
            acc[q] = make_float2(0.f, 0.f);
            run_pat[q] = -1;
            run_val[q] = 0.f;
        }
        for (int qb = e0; qb < e1; qb += 32) {
            const int cnt = min(32, e1 - qb);
            // entries past this chunk read as 0: no load, no contribution, no `last` bit
            // (a real entry is never 0: the only entry with parent 0 and mode 0 is
            // the single, hence last, entry of state (k, 0, ..., 0))
            const uint32_t mine = lane < cnt ? __ldg(t.entries + qb + lane) : 0u;
            const int nb = (cnt + 7) >> 3;
            for (int r0 = 0; r0 < 8 * nb; r0 += 8) {
                uint32_t e[8];
                float2 v[8][GPW];
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    e[r] = __shfl_sync(0xffffffffu, mine, r0 + r);
                    const uint32_t off = (e[r] >> 6) << 5;  // parent rank * 32 (elements)
#pragma unroll
                    for (int q = 0; q < GPW; ++q) {
                        v[r][q] = make_float2(0.f, 0.f);
                        if (e[r] != 0u) v[r][q] = first_layer ? make_float2(1.f, 0.f) : __ldg(prevg[q] + off);
                    }
                }
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const uint32_t uoff = (e[r] << 7) & 0x1F00u;  // mode * 256 bytes
#pragma unroll
                    for (int q = 0; q < GPW; ++q) {
                        const float2 uu = *reinterpret_cast<const float2 *>(usb + q * kUsGroup + uoff);
                        acc[q] = cfma(uu, v[r][q], acc[q]);
                    }
                    if (e[r] & 1u) {
                        // child c0 + ci is complete
                        const int64_t c = c0 + ci;
                        const float w = (EPI != EPI_STORE) ? __shfl_sync(0xffffffffu, wl, ci) : 0.f;
                        const int pat = (EPI == EPI_THRESH) ? __shfl_sync(0xffffffffu, patl, ci) : 0;
#pragma unroll
                        for (int q = 0; q < GPW; ++q) {
                            if (SAVE || EPI == EPI_STORE) {
                                if (grp0 + q < a.NG) nextg[q][(uint32_t)c << 5] = acc[q];
                            }
                            if (EPI == EPI_PROBS) {
                                tile[(q * 32 + lane) * 33 + ci] = w * (acc[q].x * acc[q].x + acc[q].y * acc[q].y);
                            } else if (EPI == EPI_AMPS) {
                                reinterpret_cast<float2 *>(tile)[(q * 32 + lane) * 33 + ci] = cscale(acc[q], sqrtf(w));
                            } else if (EPI == EPI_THRESH) {
                                const float pr = w * (acc[q].x * acc[q].x + acc[q].y * acc[q].y);
                                if (pat != run_pat[q]) {
                                    if (run_pat[q] >= 0 && valid[q])
                                        atomicAdd(reinterpret_cast<float *>(a.out) + (int64_t)inst[q] * a.K + run_pat[q],
                                                  run_val[q]);
                                    run_pat[q] = pat;
                                    run_val[q] = 0.f;
                                }
                                run_val[q] += pr;
                            }
                            acc[q] = make_float2(0.f, 0.f);
                        }
                        ++ci;
                    }
                }
            }
        }
        if (EPI == EPI_THRESH) {
#pragma unroll
            for (int q = 0; q < GPW; ++q)
                if (run_pat[q] >= 0 && valid[q])
                    atomicAdd(reinterpret_cast<float *>(a.out) + (int64_t)inst[q] * a.K + run_pat[q], run_val[q]);
        }
        if (EPI == EPI_PROBS || EPI == EPI_AMPS) {
            __syncwarp();
#pragma unroll
            for (int q = 0; q < GPW; ++q) {
                for (int i = 0; i < kLanes; ++i) {
                    const int ii = (grp0 + q) * kLanes + i;
                    if (grp0 + q < a.NG && ii < a.B && lane < nc) {
                        if (EPI == EPI_PROBS) {
                            reinterpret_cast<float *>(a.out)[(int64_t)ii * a.K + c0 + lane] = tile[(q * 32 + i) * 33 + lane];
                        } else {
                            reinterpret_cast<float2 *>(a.out)[(int64_t)ii * a.K + c0 + lane] =
                                reinterpret_cast<const float2 *>(tile)[(q * 32 + i) * 33 + lane];
                        }
                    }
                }
            }
            __syncwarp();
        }
    }
}

template <int GPW>
static size_t tab_smem(int epi) {
    return GPW * fwd_smem_bytes(epi);
}

template <int GPW>
static cudaError_t tab_attrs() {
    cudaError_t e;
    const int sp = (int)tab_smem<GPW>(EPI_PROBS), sa = (int)tab_smem<GPW>(EPI_AMPS);
    if ((e = cudaFuncSetAttribute(slos_fwd_tab_kernel<EPI_PROBS, false, GPW>, cudaFuncAttributeMaxDynamicSharedMemorySize, sp)))
        return e;
    if ((e = cudaFuncSetAttribute(slos_fwd_tab_kernel<EPI_PROBS, true, GPW>, cudaFuncAttributeMaxDynamicSharedMemorySize, sp)))
        return e;
    if ((e = cudaFuncSetAttribute(slos_fwd_tab_kernel<EPI_AMPS, false, GPW>, cudaFuncAttributeMaxDynamicSharedMemorySize, sa)))
        return e;
    return cudaFuncSetAttribute(slos_fwd_tab_kernel<EPI_AMPS, true, GPW>, cudaFuncAttributeMaxDynamicSharedMemorySize, sa);
}

cudaError_t slos_tab_init() { return tab_attrs<1>(); }

template <int GPW>
static cudaError_t launch_tab(const FwdArgs &a, const TabArgs &t, int epi, bool save, int blocks_x, cudaStream_t s) {
    dim3 grid(blocks_x, (a.NG + GPW - 1) / GPW);
    const size_t sm = tab_smem<GPW>(epi);
    switch (epi * 2 + (save ? 1 : 0)) {
        case 0:
        case 1: slos_fwd_tab_kernel<EPI_STORE, true, GPW><<<grid, kThreads, 0, s>>>(a, t); break;
        case 2: slos_fwd_tab_kernel<EPI_PROBS, false, GPW><<<grid, kThreads, sm, s>>>(a, t); break;
        case 3: slos_fwd_tab_kernel<EPI_PROBS, true, GPW><<<grid, kThreads, sm, s>>>(a, t); break;
        case 4: slos_fwd_tab_kernel<EPI_AMPS, false, GPW><<<grid, kThreads, sm, s>>>(a, t); break;
        case 5: slos_fwd_tab_kernel<EPI_AMPS, true, GPW><<<grid, kThreads, sm, s>>>(a, t); break;
        case 6: slos_fwd_tab_kernel<EPI_THRESH, false, GPW><<<grid, kThreads, 0, s>>>(a, t); break;
        case 7: slos_fwd_tab_kernel<EPI_THRESH, true, GPW><<<grid, kThreads, 0, s>>>(a, t); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// One instance group per warp: serving two groups from one entry stream
// (GPW = 2) halves the entry traffic but measured slower on GB300 (register
// pressure), so only GPW = 1 is instantiated.
cudaError_t slos_launch_fwd_tab(const FwdArgs &a, const TabArgs &t, int epi, bool save, int blocks_x, cudaStream_t s) {
    return launch_tab<1>(a, t, epi, save, blocks_x, s);
}

}  // namespace slos
