// Amplitude-encoded input (Sec. II-C, amplitude encoding): the input is a
// state vector |x> = sum_s x_s |s> over the plan's basis (n photons), the
// output is U|x>, with amplitudes
//     psi(t) = sum_s <t|U|s> x_s = sum_s Phi[t][s] x_s,
// Phi the n-photon transfer matrix of U.  Phi is built layer by layer with
// the photon-by-photon recursion of Sec. II-A.2/II-A.3 applied to every input
// column at once: for a k-photon input s with highest occupied mode c,
//     A_k[s][t] = sum_{j : t_j > 0} U[j][c] A_{k-1}[s - e_c][t - e_j],
// A_0 = 1, so A_n[s][t] = Per(U[rows t, cols s]) / prod t!, and
// <t|U|s> = A_n[s][t] sqrt(prod t!) / sqrt(prod s!).  The rows t use the
// plan's fixed-width parent slots; the columns a per-state (s - e_c, c)
// table.  Then one complex GEMM applies Phi to every input vector of the
// batch (U is shared by the batch, as the layer's weights are).
//
// The GEMM runs on the tensor cores as one real GEMM with K' = 2K:
//     [Yr | Yi](b, t) = sum_s  xr_s [Ar | Ai](s, t) + xi_s [-Ai | Ar](s, t),
// x_s = X[b][s] / g_s, A = A_n, its output columns interleaved (2t = re,
// 2t + 1 = im of output t) so the epilogue forms g_t (Yr + i Yi) and its
// |.|^2 from adjacent columns of one row.  For FP32-accurate products in TF32
// (the tensor core reads 10 mantissa bits) every operand value v is split
// into hi = v rounded to TF32 and lo = v - hi, and the GEMM sums
// A_hi B_hi + A_hi B_lo + A_lo B_hi (the three-product split-precision
// scheme; the dropped lo lo term is ~2^-22 of the product), accumulating in
// FP32, in chunks of 32 MMAs in tensor memory whose sums the epilogue adds
// in FP32 registers with round-to-nearest (tc_gemm_chunked_kernel: the
// tensor core's own accumulation over the whole K biased |psi|^2 low by
// 4e-5).  The batch runs in chunks of kEncodeChunk rows, so the split copy of
// X needs a fixed workspace.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "../../include/slos.h"
#include "common.cuh"
#include "plan.h"
#include "profile.h"
#include "tab_launch.h"
#include "tc_gemm.cuh"

namespace slos {
slos_status_t fail(slos_status_t st, const std::string &msg);

constexpr int kTransferThreads = 256;

template <int KW>
__global__ void __launch_bounds__(kTransferThreads)
    transfer_kernel(const float2 *U, int m, const uint32_t *slots, const uint32_t *colinfo, int64_t Fk, int64_t Fp,
                    const float2 *prev, float2 *cur, int first) {
    __shared__ float2 uc[32];  // column c of U, zero past m (padding slots name mode kMaxModes)
    const int64_t s = blockIdx.y;
    const uint32_t ci = __ldg(colinfo + s);
    const int c = (int)(ci & 31u);
    const int64_t sp = ci >> 5;
    if (threadIdx.x < 32) uc[threadIdx.x] = (int)threadIdx.x < m ? U[threadIdx.x * m + c] : make_float2(0.f, 0.f);
    __syncthreads();
    const int64_t t = (int64_t)blockIdx.x * kTransferThreads + threadIdx.x;
    if (t >= Fk) return;
    uint32_t e[KW];
    const uint4 *sl = reinterpret_cast<const uint4 *>(slots) + t * (KW / 4);
#pragma unroll
    for (int q4 = 0; q4 < KW / 4; ++q4) {
        const uint4 w4 = __ldg(sl + q4);
        e[4 * q4] = w4.x;
        e[4 * q4 + 1] = w4.y;
        e[4 * q4 + 2] = w4.z;
        e[4 * q4 + 3] = w4.w;
    }
    float2 acc;
    if (first) {
        acc = uc[e[0] & 31u];  // one photon: <e_j|U|e_c> = U[j][c]
    } else {
        const float2 *pv = prev + sp * Fp;
        acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < KW; ++q) acc = cfma(uc[e[q] & 31u], pv[e[q] >> 5], acc);
    }
    cur[s * Fk + t] = acc;
}

// TF32 split of an FP32 value: hi = v rounded to nearest TF32 (ties away),
// lo = v - hi (exact in FP32).
__device__ __forceinline__ void tf32_split(float v, float &hi, float &lo) {
    uint32_t h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
    hi = __uint_as_float(h);
    lo = v - hi;
}

constexpr int kEncodeChunk = 4096;  // batch rows per GEMM launch
constexpr int kEncodeKAlign = 32;   // K' padded to whole 128-byte TF32 stage rows

// Real-form operand B of the GEMM, [N = 2K rows][K2 cols], K-major:
//   row 2t:     cols s -> Ar[s][t],  K + s -> -Ai[s][t]
//   row 2t + 1: cols s -> Ai[s][t],  K + s ->  Ar[s][t]
// split into hi and lo copies; 32 x 32 tiles of A through shared memory, so
// both the read (along t) and the writes (along s) are coalesced.
__global__ void __launch_bounds__(256) encode_split_b_kernel(const float2 *A, int64_t K, int64_t K2, float *bhi,
                                                             float *blo) {
    __shared__ float2 tile[32][33];
    const int64_t s0 = (int64_t)blockIdx.y * 32, t0 = (int64_t)blockIdx.x * 32;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int64_t ss = s0 + i, tt = t0 + threadIdx.x;
        tile[i][threadIdx.x] = (ss < K && tt < K) ? A[ss * K + tt] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int64_t tt = t0 + i, ss = s0 + threadIdx.x;
        if (tt >= K || ss >= K) continue;
        const float2 v = tile[threadIdx.x][i];  // A[ss][tt]
        const float vals[4] = {v.x, -v.y, v.y, v.x};  // (2t, s), (2t, K+s), (2t+1, s), (2t+1, K+s)
        const int64_t o[4] = {2 * tt * K2 + ss, 2 * tt * K2 + K + ss, (2 * tt + 1) * K2 + ss, (2 * tt + 1) * K2 + K + ss};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float h, l;
            tf32_split(vals[q], h, l);
            bhi[o[q]] = h;
            blo[o[q]] = l;
        }
    }
}

// Real-form operand A of the GEMM for batch rows [b0, b0 + rows):
// [rows][K2], cols s -> Re X[b][s] / g_s, K + s -> Im X[b][s] / g_s, the
// padding columns 2K .. K2-1 zero; split into hi and lo copies.
__global__ void __launch_bounds__(256) encode_split_a_kernel(const float2 *X, const float *g, int64_t b0, int rows,
                                                             int64_t K, int64_t K2, float *ahi, float *alo) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)rows * K2) return;
    const int64_t r = i / K2, c = i % K2;
    float v = 0.f;
    if (c < 2 * K) {
        const int64_t ss = c < K ? c : c - K;
        const float2 x = X[(b0 + r) * K + ss];
        v = (c < K ? x.x : x.y) / __ldg(g + ss);
    }
    float h, l;
    tf32_split(v, h, l);
    ahi[i] = h;
    alo[i] = l;
}

// FP32 matrix [rows][cols] (row stride ld elements, a multiple of 4), box
// 32 x box_rows, 128-byte swizzle: the TF32 operand layout of tc_gemm.cuh.
static PFN_cuTensorMapEncodeTiled_v12000 encode_map_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *q = nullptr;
        cudaDriverEntryPointQueryResult r;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &q, 12000, cudaEnableDefault, &r) ==
                cudaSuccess &&
            r == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(q);
    });
    return fn;
}
static bool make_map_f32(CUtensorMap *map, const float *ptr, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
    auto fn = encode_map_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
    cuuint32_t box[2] = {(cuuint32_t)tc::TcKind<1>::kElems, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(ptr), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static bool encodable(const slos_plan_s *p) {
    if (!p->tab.enabled || !p->tab.gfact || p->K > kMaxEncodeStates) return false;
    for (int k = 1; k <= p->n; ++k)
        if (!p->tab.layer[k].colinfo) return false;
    return true;
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

static int64_t encode_k2(const slos_plan_s *p) {
    return (2 * p->K + kEncodeKAlign - 1) / kEncodeKAlign * kEncodeKAlign;
}

// workspace: the transfer matrices of layers n and n-1, then the split
// operands B_hi, B_lo [2K][K2] and A_hi, A_lo [kEncodeChunk][K2]
static size_t encode_bytes(const slos_plan_s *p) {
    const int n = p->n;
    const size_t a = (size_t)p->F[n] * p->F[n] * sizeof(float2);
    const size_t b = n >= 2 ? (size_t)p->F[n - 1] * p->F[n - 1] * sizeof(float2) : 0;
    const size_t bs = (size_t)2 * p->K * encode_k2(p) * sizeof(float);
    const size_t as = (size_t)kEncodeChunk * encode_k2(p) * sizeof(float);
    return align256(a) + align256(b) + 2 * align256(bs) + 2 * align256(as);
}

}  // namespace slos

using namespace slos;

extern "C" {

slos_status_t slos_encoded_workspace_bytes(slos_plan_t p, size_t *bytes) {
    if (!p || p->kind != 0 || !bytes) return fail(SLOS_ERR_INVALID_ARG, "slos_encoded_workspace_bytes: bad argument");
    if (!encodable(p))
        return fail(SLOS_ERR_UNSUPPORTED, "slos_encoded_workspace_bytes: amplitude encoding needs a PNR plan with at "
                                          "most 32768 outputs");
    *bytes = encode_bytes(p);
    return SLOS_OK;
}

slos_status_t slos_encoded_forward(slos_plan_t p, const void *U, const void *X, int batch, slos_output_t output,
                                   void *out, void *workspace, size_t workspace_bytes, void *stream) {
    if (!p || p->kind != 0) return fail(SLOS_ERR_INVALID_ARG, "slos_encoded_forward: not a single-shape plan");
    if (!encodable(p))
        return fail(SLOS_ERR_UNSUPPORTED, "slos_encoded_forward: amplitude encoding needs a PNR plan with at most "
                                          "32768 outputs");
    if (batch < 0) return fail(SLOS_ERR_INVALID_ARG, "slos_encoded_forward: negative batch");
    if (output != SLOS_OUT_PROBS && output != SLOS_OUT_AMPS)
        return fail(SLOS_ERR_INVALID_ARG, "slos_encoded_forward: bad output");
    if (!U || (batch > 0 && (!X || !out))) return fail(SLOS_ERR_INVALID_ARG, "slos_encoded_forward: NULL pointer");
    if (!workspace || workspace_bytes < encode_bytes(p))
        return fail(SLOS_ERR_INVALID_ARG, "slos_encoded_forward: workspace too small (slos_encoded_workspace_bytes)");
    cudaStream_t s = (cudaStream_t)stream;
    const int n = p->n, m = p->m;
    char *ws = reinterpret_cast<char *>(workspace);
    float2 *buf[2] = {reinterpret_cast<float2 *>(ws),
                      reinterpret_cast<float2 *>(ws + align256((size_t)p->F[n] * p->F[n] * sizeof(float2)))};
    const float2 *Ud = reinterpret_cast<const float2 *>(U);
    cudaError_t e;
    {
        ProfScope ps("slos_transfer", 0.0, s);
        for (int k = 1; k <= n; ++k) {
            const int64_t Fk = p->F[k], Fp = p->F[k - 1];
            float2 *cur = buf[(n - k) & 1];
            const float2 *prev = k >= 2 ? buf[(n - k + 1) & 1] : nullptr;
            dim3 grid((unsigned)((Fk + kTransferThreads - 1) / kTransferThreads), (unsigned)Fk);
            const uint32_t *sl = p->tab.layer[k].slots, *ci = p->tab.layer[k].colinfo;
            switch (p->tab.layer[k].kw) {
                case 4: transfer_kernel<4><<<grid, kTransferThreads, 0, s>>>(Ud, m, sl, ci, Fk, Fp, prev, cur, k == 1); break;
                case 8: transfer_kernel<8><<<grid, kTransferThreads, 0, s>>>(Ud, m, sl, ci, Fk, Fp, prev, cur, k == 1); break;
                default: transfer_kernel<12><<<grid, kTransferThreads, 0, s>>>(Ud, m, sl, ci, Fk, Fp, prev, cur, k == 1); break;
            }
            if ((e = cudaGetLastError()) != cudaSuccess)
                return fail(SLOS_ERR_CUDA, std::string("slos_encoded_forward: ") + cudaGetErrorString(e));
        }
    }
    if (batch == 0) return SLOS_OK;
    const int64_t K = p->K, K2 = encode_k2(p);
    const size_t bs = (size_t)2 * K * K2 * sizeof(float), as = (size_t)kEncodeChunk * K2 * sizeof(float);
    char *w = ws + align256((size_t)p->F[n] * p->F[n] * sizeof(float2)) +
              (n >= 2 ? align256((size_t)p->F[n - 1] * p->F[n - 1] * sizeof(float2)) : 0);
    float *bhi = reinterpret_cast<float *>(w), *blo = reinterpret_cast<float *>(w + align256(bs));
    float *ahi = reinterpret_cast<float *>(w + 2 * align256(bs));
    float *alo = reinterpret_cast<float *>(w + 2 * align256(bs) + align256(as));
    {
        ProfScope ps("slos_encode_split", 0.0, s);
        // B's padding columns stay zero: clear both copies, then fill
        if ((e = cudaMemsetAsync(bhi, 0, 2 * align256(bs), s)) != cudaSuccess)
            return fail(SLOS_ERR_CUDA, std::string("slos_encoded_forward: ") + cudaGetErrorString(e));
        dim3 grid((unsigned)((K + 31) / 32), (unsigned)((K + 31) / 32));
        encode_split_b_kernel<<<grid, dim3(32, 8), 0, s>>>(buf[0], K, K2, bhi, blo);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return fail(SLOS_ERR_CUDA, std::string("slos_encoded_forward: ") + cudaGetErrorString(e));
    }
    static bool attr_done[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_done[dev]) {
        if ((e = cudaFuncSetAttribute(tc::tc_gemm_chunked_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      tc::kCkSmem)) != cudaSuccess)
            return fail(SLOS_ERR_CUDA, std::string("slos_encoded_forward: ") + cudaGetErrorString(e));
        attr_done[dev] = true;
    }
    CUtensorMap mah, mal, mbh, mbl;
    if (!make_map_f32(&mbh, bhi, 2 * K, K2, K2, tc::kCkBN) || !make_map_f32(&mbl, blo, 2 * K, K2, K2, tc::kCkBN) ||
        !make_map_f32(&mah, ahi, kEncodeChunk, K2, K2, tc::BM) || !make_map_f32(&mal, alo, kEncodeChunk, K2, K2, tc::BM))
        return fail(SLOS_ERR_CUDA, "slos_encoded_forward: cuTensorMapEncodeTiled failed");
    const float2 *Xd = reinterpret_cast<const float2 *>(X);
    for (int b0 = 0; b0 < batch; b0 += kEncodeChunk) {
        const int rows = std::min(kEncodeChunk, batch - b0);
        {
            ProfScope ps("slos_encode_split", 0.0, s);
            const int64_t cnt = (int64_t)rows * K2;
            encode_split_a_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(Xd, p->tab.gfact, b0, rows, K, K2,
                                                                                 ahi, alo);
            if ((e = cudaGetLastError()) != cudaSuccess)
                return fail(SLOS_ERR_CUDA, std::string("slos_encoded_forward: ") + cudaGetErrorString(e));
        }
        tc::TcArgs g;
        memset(&g, 0, sizeof(g));
        g.M = rows;
        g.N = (int)(2 * K);
        g.K = (int)K2;
        g.ldc = (int)K;
        g.C = output == SLOS_OUT_AMPS ? (void *)(reinterpret_cast<float2 *>(out) + (int64_t)b0 * K)
                                      : (void *)(reinterpret_cast<float *>(out) + (int64_t)b0 * K);
        g.colscale = p->tab.gfact;
        g.amps = output == SLOS_OUT_AMPS ? 1 : 0;
        g.err = p->d_status + 2;
        const int64_t tiles = (int64_t)((g.N + tc::kCkBN - 1) / tc::kCkBN) * ((rows + tc::BM - 1) / tc::BM);
        const unsigned grid = (unsigned)std::min<int64_t>(tiles, p->sm_count);
        ProfScope ps("slos_encode_gemm", 3.0 * 2.0 * rows * (double)g.N * (double)K2, s);  // flops
        tc::tc_gemm_chunked_kernel<<<grid, tc::kCkThreads, tc::kCkSmem, s>>>(mah, mbh, mal, mbl, g);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return fail(SLOS_ERR_CUDA, std::string("slos_encoded_forward: ") + cudaGetErrorString(e));
    }
    return SLOS_OK;
}

}  // extern "C"
