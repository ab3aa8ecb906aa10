// Tensor-core GEMM for sm_103a: C[M][N] = A[M][K] . B[N][K]^T, BF16 inputs
// (both K-major), FP32 accumulation in tensor memory (TMEM), fused epilogues.
// tc_gemm_chunked_kernel (end of the file) takes TF32 operands (FP32
// storage, the tensor core reads 19 bits of each): a stage row is 128 bytes
// either way (64 BF16 or 32 FP32 elements), four MMAs of 32 bytes of K each
// (K = 16 or 8), so the ring, the swizzle and the descriptors are the same.
// Two kernels share the pipeline below: tc_gemm_kernel (one tile per CTA) and
// tc_gemm_persist_kernel (one CTA per SM over many tiles, two accumulators,
// the epilogue of one tile overlapping the next tile's MMAs), which the
// library launches.
//
// One CTA = 128 threads computes one 128 x 256 output tile.
//   warp 0, lane 0: TMA producer.  cp.async.bulk.tensor loads 128x64 tiles of
//                   A and B (128-byte swizzle) into a 4-stage ring; each stage
//                   has a `full` mbarrier (transaction bytes) and an `empty`
//                   mbarrier (arrived by tcgen05.commit when the MMAs that
//                   read the stage are done).
//   warp 1, lane 0: MMA issuer.  Four tcgen05.mma.kind::f16 (K = 16 each) per
//                   stage into one 128 x 256 FP32 accumulator in TMEM
//                   (256 of the SM's 512 TMEM columns).
//   all 4 warps:    epilogue.  tcgen05.ld 32x32b: warp w reads TMEM lanes
//                   32w..32w+31 (= output rows), 16 columns per load.
// Every mbarrier wait has an iteration limit; a wait that runs out sets the
// error word, the CTA still frees its TMEM and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace slos {
namespace tc {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int A_TILE = BM * BK * 2;  // bytes
constexpr int B_TILE = BN * BK * 2;
constexpr int STAGE_BYTES = A_TILE + B_TILE;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
constexpr uint32_t TMEM_COLS = BN;
constexpr long long kWaitLimit = 1ll << 22;  // tries; a few seconds at most

enum TcEpi : int {
    TC_F32 = 0,        // C = acc                         (float)
    TC_F32_BIAS = 1,   // C = acc + bias[n]               (float)
    TC_GELU = 2,       // Z = acc + bias[n] (bf16, aux), C = gelu(Z) (bf16)
    TC_GELU_BWD = 3,   // C = acc * gelu'(Z), Z = aux (bf16 in), C bf16
    TC_F32_ACCUM = 4,  // C += acc                        (float)
    TC_ENCODE = 5,     // columns (2t, 2t+1) = (re, im) of output t: psi = colscale[t] (re + i im);
                       //   C float |psi|^2, or complex64 psi when amps (row stride ldc outputs)
};

struct TcArgs {
    int M, N, K;
    void *C;              // [M][ldc]
    int ldc;
    const float *bias;    // [N]
    __nv_bfloat16 *aux;   // [M][ldc] (Z for TC_GELU out, TC_GELU_BWD in)
    int *err;             // error word (device)
    const float *colscale;  // TC_ENCODE: [N / 2]
    int amps;               // TC_ENCODE: complex64 output
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Bounded wait: true if the phase completed, false if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (long long i = 0; i < kWaitLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor, K-major operand with 128-byte swizzle:
// start address >> 4 (bits 0-13), leading byte offset 16 B (unused for this
// layout, bits 16-29), stride byte offset 1024 B between 8-row groups
// (bits 32-45), fixed 0b001 (bits 46-48), swizzle mode 2 = 128 B (bits 61-63).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), A and B
// BF16 (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 (bits 17-22),
// M >> 4 (bits 24-28).
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
        : "memory");
}
// Operand kinds: 0 = BF16, 1 = TF32; elements per 128-byte stage row.
template <int KIND>
struct TcKind {
    static constexpr int kElems = KIND == 0 ? 64 : 32;
};

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// GELU, tanh form, and its derivative (the surrogate's activation).
__device__ __forceinline__ float gelu_f(float z) {
    const float c = 0.7978845608028654f;  // sqrt(2/pi)
    const float u = c * (z + 0.044715f * z * z * z);
    return 0.5f * z * (1.f + tanhf(u));
}
__device__ __forceinline__ float gelu_grad(float z) {
    const float c = 0.7978845608028654f;
    const float u = c * (z + 0.044715f * z * z * z);
    const float t = tanhf(u);
    return 0.5f * (1.f + t) + 0.5f * z * (1.f - t * t) * c * (1.f + 3.f * 0.044715f * z * z);
}

// Epilogue of one 16-column segment of an output row: v holds the
// accumulator values of row `row`, columns col0 .. col0 + 15.
template <int EPI>
__device__ __forceinline__ void tc_store16(const TcArgs &g, int row, int col0, float (&v)[16], bool vec) {
    if (EPI == TC_ENCODE) {
        if (row < g.M) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int t = col0 / 2 + i;
                if (2 * t >= g.N) break;
                const float c = g.colscale[t];
                const float re = v[2 * i] * c, im = v[2 * i + 1] * c;
                const int64_t o = (int64_t)row * g.ldc + t;
                if (g.amps) reinterpret_cast<float2 *>(g.C)[o] = make_float2(re, im);
                else reinterpret_cast<float *>(g.C)[o] = re * re + im * im;
            }
        }
        return;
    }
    if (row < g.M && col0 < g.N) {
        const int64_t o0 = (int64_t)row * g.ldc + col0;
        if (EPI == TC_F32_BIAS || EPI == TC_GELU) {
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] += (col0 + i < g.N) ? g.bias[col0 + i] : 0.f;
        }
        if (vec && col0 + 16 <= g.N) {
            if (EPI == TC_F32 || EPI == TC_F32_BIAS || EPI == TC_F32_ACCUM) {
                float4 *dst = reinterpret_cast<float4 *>(reinterpret_cast<float *>(g.C) + o0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float4 w = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                    if (EPI == TC_F32_ACCUM) {
                        const float4 old = dst[q];
                        w.x += old.x;
                        w.y += old.y;
                        w.z += old.z;
                        w.w += old.w;
                    }
                    dst[q] = w;
                }
            } else {
                __align__(16) __nv_bfloat16 out[16];
                if (EPI == TC_GELU) {
                    __align__(16) __nv_bfloat16 zb[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        zb[i] = __float2bfloat16(v[i]);
                        out[i] = __float2bfloat16(gelu_f(__bfloat162float(zb[i])));
                    }
                    uint4 *za = reinterpret_cast<uint4 *>(g.aux + o0);
                    za[0] = reinterpret_cast<const uint4 *>(zb)[0];
                    za[1] = reinterpret_cast<const uint4 *>(zb)[1];
                } else {  // TC_GELU_BWD
                    __align__(16) __nv_bfloat16 zb[16];
                    const uint4 *zs = reinterpret_cast<const uint4 *>(g.aux + o0);
                    reinterpret_cast<uint4 *>(zb)[0] = zs[0];
                    reinterpret_cast<uint4 *>(zb)[1] = zs[1];
#pragma unroll
                    for (int i = 0; i < 16; ++i) out[i] = __float2bfloat16(v[i] * gelu_grad(__bfloat162float(zb[i])));
                }
                uint4 *dst = reinterpret_cast<uint4 *>(reinterpret_cast<__nv_bfloat16 *>(g.C) + o0);
                dst[0] = reinterpret_cast<const uint4 *>(out)[0];
                dst[1] = reinterpret_cast<const uint4 *>(out)[1];
            }
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int col = col0 + i;
                if (col >= g.N) break;
                const int64_t o = o0 + i;
                const float x = v[i];
                if (EPI == TC_F32 || EPI == TC_F32_BIAS) {
                    reinterpret_cast<float *>(g.C)[o] = x;
                } else if (EPI == TC_F32_ACCUM) {
                    reinterpret_cast<float *>(g.C)[o] += x;
                } else if (EPI == TC_GELU) {
                    const __nv_bfloat16 zb = __float2bfloat16(x);
                    g.aux[o] = zb;
                    reinterpret_cast<__nv_bfloat16 *>(g.C)[o] = __float2bfloat16(gelu_f(__bfloat162float(zb)));
                } else {  // TC_GELU_BWD
                    const float z = __bfloat162float(g.aux[o]);
                    reinterpret_cast<__nv_bfloat16 *>(g.C)[o] = __float2bfloat16(x * gelu_grad(z));
                }
            }
        }
    }
}

template <int EPI>
__global__ void __launch_bounds__(128, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, TcArgs g) {
    extern __shared__ uint8_t smem_tc[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_tc) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = base;
    uint8_t *sB = base + STAGES * A_TILE;
    uint64_t *full = reinterpret_cast<uint64_t *>(sB + STAGES * B_TILE);
    uint64_t *empty = full + STAGES;
    uint64_t *done = empty + STAGES;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int nk = (g.K + BK - 1) / BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer
        int issued = 0;
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % STAGES;
            const uint32_t ph = (kt / STAGES) & 1;
            if (kt >= STAGES && !mbar_wait(empty + s, ph ^ 1)) {
                atomicExch(g.err, 1);
                *abort_flag = 1;
                break;
            }
            if (*abort_flag) break;
            mbar_expect_tx(full + s, STAGE_BYTES);
            tma_load_2d(sA + s * A_TILE, &ta, kt * BK, m0, full + s);
            tma_load_2d(sB + s * B_TILE, &tb, kt * BK, n0, full + s);
            issued = kt + 1;
        }
        // never leave with copies in flight: wait (bounded) for the last loads
        for (int kt = (issued > STAGES ? issued - STAGES : 0); kt < issued; ++kt)
            mbar_wait(full + (kt % STAGES), (kt / STAGES) & 1);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % STAGES;
            const uint32_t ph = (kt / STAGES) & 1;
            if (*abort_flag || !mbar_wait(full + s, ph)) {
                atomicExch(g.err, 2);
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA + s * A_TILE), b0 = smem_u32(sB + s * B_TILE);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
                mma_bf16(tmem, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), (kt > 0 || kk > 0) ? 1u : 0u);
            mma_commit(empty + s);
        }
        mma_commit(done);  // arrives once every MMA issued above has completed
    }
    __syncwarp();
    // epilogue
    const bool ok = __all_sync(0xffffffffu, mbar_wait(done, 0) && !*abort_flag);
    if (!ok && lane == 0) atomicExch(g.err, 3);
    tc_fence_after();
    const int row = m0 + warp * 32 + lane;
    if (ok) {
        // 16 consecutive outputs per thread per TMEM load: one row segment,
        // written with 16-byte stores when the row stride allows it
        const bool vec = (g.ldc % 8) == 0;
#pragma unroll 1
        for (int c = 0; c < BN; c += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
            tc_store16<EPI>(g, row, n0 + c, v, vec);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}


// Persistent variant: one CTA per SM walks the output tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ... (row-major over 128 x 256 tiles, so the CTAs
// running together share A rows in L2).  Six warps:
//   warp 0, lane 0: TMA producer over one stage ring that runs on across tiles;
//   warp 1, lane 0: MMA issuer, alternating between two 128 x 256 FP32
//                   accumulators in TMEM (all 512 columns): tile j uses
//                   accumulator j & 1, after the epilogue has released it
//                   (`tempty`, one arrival per epilogue warp), and commits
//                   `tfull` when its last MMA has completed;
//   warps 2-5:      epilogue; warp w reads TMEM lanes 32 (w % 4) .. + 31, the
//                   quarter its position in the warpgroup gives access to.
// So a tile's epilogue runs while the next tile's loads and MMAs proceed, and
// the ring's fill is paid once per CTA.  Waits are bounded as above; a wait
// that runs out sets the error word and the abort flag, and every role leaves
// its loop.
constexpr int kPersistThreads = 192;
constexpr uint32_t kPersistTmemCols = 2 * BN;

template <int EPI>
__global__ void __launch_bounds__(kPersistThreads, 1)
    tc_gemm_persist_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, TcArgs g) {
    extern __shared__ uint8_t smem_tc[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_tc) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = base;
    uint8_t *sB = base + STAGES * A_TILE;
    uint64_t *full = reinterpret_cast<uint64_t *>(sB + STAGES * B_TILE);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;  // [2]
    uint64_t *tempty = tfull + 2;      // [2]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tempty + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = (g.K + BK - 1) / BK;
    const int ntn = (g.N + BN - 1) / BN;
    const int ntiles = ((g.M + BM - 1) / BM) * ntn;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(tfull + a, 1);
            mbar_init(tempty + a, 4);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kPersistTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // producer
            uint32_t it = 0;
            for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
                const int m0 = (t / ntn) * BM, n0 = (t % ntn) * BN;
                for (int kt = 0; kt < nk; ++kt, ++it) {
                    const int s = it % STAGES;
                    const uint32_t ph = (it / STAGES) & 1;
                    if (it >= STAGES && !mbar_wait(empty + s, ph ^ 1)) {
                        atomicExch(g.err, 1);
                        *abort_flag = 1;
                        break;
                    }
                    if (*abort_flag) break;
                    mbar_expect_tx(full + s, STAGE_BYTES);
                    tma_load_2d(sA + s * A_TILE, &ta, kt * BK, m0, full + s);
                    tma_load_2d(sB + s * B_TILE, &tb, kt * BK, n0, full + s);
                }
            }
            // never leave with copies in flight: wait (bounded) for the last loads
            for (uint32_t q = (it > (uint32_t)STAGES ? it - STAGES : 0); q < it; ++q)
                mbar_wait(full + (q % STAGES), (q / STAGES) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer
            uint32_t it = 0;
            int j = 0;
            for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, ++j) {
                const int acc = j & 1;
                const int use = j >> 1;  // this accumulator's use count
                if (use > 0 && !mbar_wait(tempty + acc, (use - 1) & 1)) {
                    atomicExch(g.err, 4);
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(acc * BN);
                for (int kt = 0; kt < nk; ++kt, ++it) {
                    const int s = it % STAGES;
                    const uint32_t ph = (it / STAGES) & 1;
                    if (*abort_flag || !mbar_wait(full + s, ph)) {
                        atomicExch(g.err, 2);
                        *abort_flag = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(sA + s * A_TILE), b0 = smem_u32(sB + s * B_TILE);
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk)
                        mma_bf16(d, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), (kt > 0 || kk > 0) ? 1u : 0u);
                    mma_commit(empty + s);
                }
                if (*abort_flag) break;
                mma_commit(tfull + acc);  // arrives once this tile's MMAs have completed
            }
        }
    } else {
        // epilogue warps
        const int q = warp & 3;
        const bool vec = (g.ldc % 8) == 0;
        int j = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
            const int acc = j & 1;
            const bool ok = __all_sync(0xffffffffu, !*abort_flag && mbar_wait(tfull + acc, (j >> 1) & 1));
            if (!ok) {
                if (lane == 0) {
                    atomicExch(g.err, 3);
                    *abort_flag = 1;
                }
                break;
            }
            tc_fence_after();
            const int m0 = (t / ntn) * BM, n0 = (t % ntn) * BN;
            const int row = m0 + q * 32 + lane;
            const uint32_t src = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN);
#pragma unroll 1
            for (int c = 0; c < BN; c += 16) {
                float v[16];
                tmem_ld16(src + (uint32_t)c, v);
                tc_store16<EPI>(g, row, n0 + c, v, vec);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty + acc);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kPersistTmemCols)
                     : "memory");
    }
}

}  // namespace tc
}  // namespace slos

namespace slos {
namespace tc {

// ---------------------------------------------------------------- chunked accumulation
// tc_gemm_chunked_kernel: the persistent pipeline (128 x 256 tiles) with the
// K sum taken in chunks of kChunkStages stages.  The tensor core's FP32
// accumulation does not round to nearest: over the ~1500 MMAs of a long K its
// errors pile up in one direction (measured: |psi|^2 of the amplitude-encoding
// GEMM biased low by 4e-5 at K' = 3 x 4032).  Here each chunk accumulates
// into one of two TMEM buffers while the epilogue warps move the other
// buffer's finished chunk into FP32 registers (half a row, 128 columns, per
// thread; round-to-nearest adds), so a truncation bias builds up only within
// one chunk.  Roles: warp 0 TMA producer, warp 1 MMA issuer, warps 2-9
// epilogue (TMEM lane quarter = warp % 4, columns 0-127 for warps 2-5 and
// 128-255 for warps 6-9).  Waits are bounded as above.
constexpr int kCkBN = 256;
constexpr int kCkStages = 4;
constexpr int kChunkStages = 8;  // 32 MMAs per chunk
constexpr int kCkThreads = 320;
constexpr int kCkEpiWarps = 8;
constexpr int kCkATile = BM * 128, kCkBTile = kCkBN * 128;  // bytes: 128-byte rows
constexpr int kCkStageBytes = kCkATile + kCkBTile;
constexpr int kCkSmem = kCkStages * kCkStageBytes + 1024 + 256;
constexpr uint32_t kCkTmemCols = 2 * kCkBN;
// kind::tf32: A and B TF32 (bits 7-9 = 2, 10-12 = 2), otherwise as kIdesc.
constexpr uint32_t kIdescTf32 =
    (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kCkBN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kIdescTf32), "r"(accumulate)
        : "memory");
}

// TF32 operands in three K segments, A_hi B_hi + A_hi B_lo + A_lo B_hi, each
// segment's tiles taken from the hi or lo copy of an operand (the
// three-TF32-product scheme for FP32-accurate products); TC_ENCODE epilogue.
static __global__ void __launch_bounds__(kCkThreads, 1)
    tc_gemm_chunked_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
                           const __grid_constant__ CUtensorMap ta_lo, const __grid_constant__ CUtensorMap tb_lo,
                           TcArgs g) {
    constexpr int KE = TcKind<1>::kElems;
    extern __shared__ uint8_t smem_tc[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_tc) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = base;
    uint8_t *sB = base + kCkStages * kCkATile;
    uint64_t *full = reinterpret_cast<uint64_t *>(sB + kCkStages * kCkBTile);
    uint64_t *empty = full + kCkStages;
    uint64_t *cfull = empty + kCkStages;  // [2] a chunk's MMAs are done
    uint64_t *cempty = cfull + 2;         // [2] the epilogue has taken the chunk
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(cempty + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk1 = (g.K + KE - 1) / KE;
    const int nk = 3 * nk1;
    const int nchunks = (nk + kChunkStages - 1) / kChunkStages;
    const int ntn = (g.N + kCkBN - 1) / kCkBN;
    const int ntiles = ((g.M + BM - 1) / BM) * ntn;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kCkStages; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(cfull + a, 1);
            mbar_init(cempty + a, kCkEpiWarps);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kCkTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // producer: every stage of every tile, in order
            uint32_t it = 0;
            for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
                const int m0 = (t / ntn) * BM, n0 = (t % ntn) * kCkBN;
                for (int kt = 0; kt < nk; ++kt, ++it) {
                    const int s = it % kCkStages;
                    const uint32_t ph = (it / kCkStages) & 1;
                    if (it >= (uint32_t)kCkStages && !mbar_wait(empty + s, ph ^ 1)) {
                        atomicExch(g.err, 1);
                        *abort_flag = 1;
                        break;
                    }
                    if (*abort_flag) break;
                    mbar_expect_tx(full + s, kCkStageBytes);
                    const int seg = kt / nk1;  // 0: A_hi B_hi, 1: A_hi B_lo, 2: A_lo B_hi
                    const int kx = (kt - seg * nk1) * KE;
                    tma_load_2d(sA + s * kCkATile, seg == 2 ? &ta_lo : &ta, kx, m0, full + s);
                    tma_load_2d(sB + s * kCkBTile, seg == 1 ? &tb_lo : &tb, kx, n0, full + s);
                }
            }
            for (uint32_t q = (it > (uint32_t)kCkStages ? it - kCkStages : 0); q < it; ++q)
                mbar_wait(full + (q % kCkStages), (q / kCkStages) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer: chunk c of the CTA's walk goes to buffer c & 1
            uint32_t it = 0, c = 0;
            for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
                for (int ch = 0; ch < nchunks && !*abort_flag; ++ch, ++c) {
                    const int b = c & 1;
                    const uint32_t use = c >> 1;
                    if (use > 0 && !mbar_wait(cempty + b, (use - 1) & 1)) {
                        atomicExch(g.err, 4);
                        *abort_flag = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(b * kCkBN);
                    const int k1 = min(nk, (ch + 1) * kChunkStages);
                    for (int kt = ch * kChunkStages; kt < k1; ++kt, ++it) {
                        const int s = it % kCkStages;
                        const uint32_t ph = (it / kCkStages) & 1;
                        if (*abort_flag || !mbar_wait(full + s, ph)) {
                            atomicExch(g.err, 2);
                            *abort_flag = 1;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a0 = smem_u32(sA + s * kCkATile), b0 = smem_u32(sB + s * kCkBTile);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            mma_tf32(d, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32),
                                     (kt > ch * kChunkStages || kk > 0) ? 1u : 0u);
                        mma_commit(empty + s);
                    }
                    if (*abort_flag) break;
                    mma_commit(cfull + b);
                }
            }
        }
    } else {
        // epilogue warps: each thread sums 128 columns of its row over the chunks
        constexpr int HC = kCkBN / 2;
        const int q = warp & 3;
        const int hc = (warp - 2) >> 2;  // column half
        uint32_t c = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            float acc[HC];
#pragma unroll
            for (int i = 0; i < HC; ++i) acc[i] = 0.f;
            for (int ch = 0; ch < nchunks; ++ch, ++c) {
                const int b = c & 1;
                ok = __all_sync(0xffffffffu, !*abort_flag && mbar_wait(cfull + b, (c >> 1) & 1));
                if (!ok) {
                    if (lane == 0) {
                        atomicExch(g.err, 3);
                        *abort_flag = 1;
                    }
                    break;
                }
                tc_fence_after();
                const uint32_t src = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * kCkBN + hc * HC);
#pragma unroll
                for (int c16 = 0; c16 < HC; c16 += 16) {
                    float v[16];
                    tmem_ld16(src + (uint32_t)c16, v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) acc[c16 + i] += v[i];
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(cempty + b);
            }
            if (!ok) break;
            const int m0 = (t / ntn) * BM, n0 = (t % ntn) * kCkBN + hc * HC;
            const int row = m0 + q * 32 + lane;
#pragma unroll
            for (int c16 = 0; c16 < HC; c16 += 16) {
                float v[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = acc[c16 + i];
                tc_store16<TC_ENCODE>(g, row, n0 + c16, v, false);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCkTmemCols) : "memory");
    }
}

}  // namespace tc
}  // namespace slos
