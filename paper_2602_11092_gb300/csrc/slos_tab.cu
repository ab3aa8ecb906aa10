// Forward photon-number layer driven by the plan's transition graph
// (Sec. II-A.3): a_k(t) = sum over the parent slots of t of U[j, c_k] a_{k-1}(parent).
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "slos_kernels.cuh"
#include "tab_launch.h"
#include "tables.h"

namespace slos {

// Fixed-width (ELL) parent lists: state c has KW slots (parent rank << 5 |
// mode, or kEllEmpty).  Each warp owns one group of 32 instances (lane =
// instance) and walks a chunk of 32 consecutive states, two at a time: the
// two states' slots arrive with 16-byte broadcast loads, all their parent
// gathers (coalesced 256-byte rows, predicated on the slot being used) are
// issued before any FMA, and the output is written in straight-line code.
template <int EPI, bool SAVE, int KW>
__global__ void __launch_bounds__(kThreads) slos_fwd_ell_kernel(FwdArgs a, TabArgs t) {
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

    // 64-bit group bases once; per-state offsets are 32-bit (table plans: F * 32 < 2^32)
    const float2 *prevg = a.prev + (size_t)grp * (size_t)a.Fprev * kLanes + lane;
    float2 *nextg = a.next + (size_t)grp * (size_t)a.Fk * kLanes + lane;
    const float2 *usl = &us[0][lane];
    float *tile = reinterpret_cast<float *>(smem_raw) + warp * (32 * 33 * (EPI == EPI_AMPS ? 2 : 1));
    const int64_t nchunks = (a.Fk + 31) / 32;
    const int64_t wstride = (int64_t)gridDim.x * kWarpsPerBlock;
    const bool first_layer = a.k == 1;

    for (int64_t ch = (int64_t)blockIdx.x * kWarpsPerBlock + warp; ch < nchunks; ch += wstride) {
        const int64_t c0 = ch * 32;
        const int nc = (int)min((int64_t)32, a.Fk - c0);
        float wl = 0.f;
        int patl = 0;
        if (EPI != EPI_STORE && lane < nc) {
            wl = __ldg(t.w + c0 + lane);
            if (EPI == EPI_THRESH) patl = __ldg(t.pat + c0 + lane);
        }
        int run_pat = -1;
        float run_val = 0.f;
        for (int ci = 0; ci < nc; ci += 2) {
            uint32_t e[2][KW];
            float2 v[2][KW];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const bool live = ci + h < nc;
                const uint4 *ep = reinterpret_cast<const uint4 *>(t.ell + (size_t)(c0 + ci + (live ? h : 0)) * KW);
#pragma unroll
                for (int q4 = 0; q4 < KW / 4; ++q4) {
                    const uint4 w4 = __ldg(ep + q4);
                    e[h][4 * q4 + 0] = live ? w4.x : kEllEmpty;
                    e[h][4 * q4 + 1] = live ? w4.y : kEllEmpty;
                    e[h][4 * q4 + 2] = live ? w4.z : kEllEmpty;
                    e[h][4 * q4 + 3] = live ? w4.w : kEllEmpty;
                }
#pragma unroll
                for (int q = 0; q < KW; ++q) {
                    v[h][q] = make_float2(0.f, 0.f);
                    if (e[h][q] != kEllEmpty)
                        v[h][q] = first_layer ? make_float2(1.f, 0.f) : __ldg(prevg + (e[h][q] & ~31u));
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int q = 0; q < KW; ++q) {
                    const uint32_t j = e[h][q] != kEllEmpty ? (e[h][q] & 31u) : 0u;
                    acc = cfma(usl[j * 32], v[h][q], acc);
                }
                const int cc = ci + h;
                const int64_t c = c0 + cc;
                const float w = (EPI != EPI_STORE) ? __shfl_sync(0xffffffffu, wl, cc & 31) : 0.f;
                const int pat = (EPI == EPI_THRESH) ? __shfl_sync(0xffffffffu, patl, cc & 31) : 0;
                if (cc < nc) {
                    if (SAVE || EPI == EPI_STORE) nextg[(uint32_t)c << 5] = acc;
                    if (EPI == EPI_PROBS) {
                        tile[lane * 33 + cc] = w * (acc.x * acc.x + acc.y * acc.y);
                    } else if (EPI == EPI_AMPS) {
                        reinterpret_cast<float2 *>(tile)[lane * 33 + cc] = cscale(acc, sqrtf(w));
                    } else if (EPI == EPI_THRESH) {
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

template <int KW>
static cudaError_t ell_attrs() {
    cudaError_t e;
    const int sa = (int)fwd_smem_bytes(EPI_AMPS);
    if ((e = cudaFuncSetAttribute(slos_fwd_ell_kernel<EPI_AMPS, false, KW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  sa)))
        return e;
    return cudaFuncSetAttribute(slos_fwd_ell_kernel<EPI_AMPS, true, KW>, cudaFuncAttributeMaxDynamicSharedMemorySize, sa);
}

cudaError_t slos_tab_init() {
    cudaError_t e;
    if ((e = ell_attrs<4>())) return e;
    if ((e = ell_attrs<8>())) return e;
    return ell_attrs<12>();
}

template <int KW>
static cudaError_t launch_ell(const FwdArgs &a, const TabArgs &t, int epi, bool save, int blocks_x, cudaStream_t s) {
    dim3 grid(blocks_x, a.NG);
    const size_t sm = fwd_smem_bytes(epi);
    switch (epi * 2 + (save ? 1 : 0)) {
        case 0:
        case 1: slos_fwd_ell_kernel<EPI_STORE, true, KW><<<grid, kThreads, 0, s>>>(a, t); break;
        case 2: slos_fwd_ell_kernel<EPI_PROBS, false, KW><<<grid, kThreads, sm, s>>>(a, t); break;
        case 3: slos_fwd_ell_kernel<EPI_PROBS, true, KW><<<grid, kThreads, sm, s>>>(a, t); break;
        case 4: slos_fwd_ell_kernel<EPI_AMPS, false, KW><<<grid, kThreads, sm, s>>>(a, t); break;
        case 5: slos_fwd_ell_kernel<EPI_AMPS, true, KW><<<grid, kThreads, sm, s>>>(a, t); break;
        case 6: slos_fwd_ell_kernel<EPI_THRESH, false, KW><<<grid, kThreads, 0, s>>>(a, t); break;
        case 7: slos_fwd_ell_kernel<EPI_THRESH, true, KW><<<grid, kThreads, 0, s>>>(a, t); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t slos_launch_fwd_tab(const FwdArgs &a, const TabArgs &t, int epi, bool save, int blocks_x, cudaStream_t s) {
    if (t.kw <= 4) return launch_ell<4>(a, t, epi, save, blocks_x, s);
    if (t.kw <= 8) return launch_ell<8>(a, t, epi, save, blocks_x, s);
    return launch_ell<12>(a, t, epi, save, blocks_x, s);
}

}  // namespace slos
