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
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/slos.h"
#include "common.cuh"
#include "plan.h"
#include "profile.h"
#include "tab_launch.h"

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

// out[b][t] = g_t sum_s (X[b][s] / g_s) A[s][t]   (g = sqrt(prod t!));
// 64 x 64 output tiles, 16 x 16 threads with 4 x 4 outputs each.
constexpr int kGT = 64, kGK = 16;

__global__ void __launch_bounds__(256) encode_gemm_kernel(const float2 *X, const float2 *A, const float *g, int B,
                                                          int64_t K, int probs, void *out) {
    __shared__ float2 xs[kGT][kGK + 1];
    __shared__ float2 as[kGK][kGT + 1];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 16 + tx;
    const int64_t b0 = (int64_t)blockIdx.y * kGT, t0 = (int64_t)blockIdx.x * kGT;
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
    for (int64_t k0 = 0; k0 < K; k0 += kGK) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int idx = tid + r * 256;  // 1024 = 64 x 16 elements of each tile
            const int xr = idx / kGK, xc = idx % kGK;
            const int64_t bb = b0 + xr, ss = k0 + xc;
            float2 v = make_float2(0.f, 0.f);
            if (bb < B && ss < K) v = cscale(X[bb * K + ss], 1.f / __ldg(g + ss));
            xs[xr][xc] = v;
            const int ar = idx / kGT, ac = idx % kGT;
            const int64_t sa = k0 + ar, ta = t0 + ac;
            as[ar][ac] = (sa < K && ta < K) ? A[sa * K + ta] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGK; ++kk) {
            float2 xv[4], av[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) xv[i] = xs[ty + 16 * i][kk];
#pragma unroll
            for (int j = 0; j < 4; ++j) av[j] = as[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = cfma(xv[i], av[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t bb = b0 + ty + 16 * i;
        if (bb >= B) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t tt = t0 + tx + 16 * j;
            if (tt >= K) continue;
            const float2 v = cscale(acc[i][j], __ldg(g + tt));
            if (probs) reinterpret_cast<float *>(out)[bb * K + tt] = v.x * v.x + v.y * v.y;
            else reinterpret_cast<float2 *>(out)[bb * K + tt] = v;
        }
    }
}

static bool encodable(const slos_plan_s *p) {
    if (!p->tab.enabled || !p->tab.gfact || p->K > kMaxEncodeStates) return false;
    for (int k = 1; k <= p->n; ++k)
        if (!p->tab.layer[k].colinfo) return false;
    return true;
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

static size_t encode_bytes(const slos_plan_s *p) {
    const int n = p->n;
    const size_t a = (size_t)p->F[n] * p->F[n] * sizeof(float2);
    const size_t b = n >= 2 ? (size_t)p->F[n - 1] * p->F[n - 1] * sizeof(float2) : 0;
    return align256(a) + align256(b);
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
    if (batch > 65535 * kGT) return fail(SLOS_ERR_UNSUPPORTED, "slos_encoded_forward: batch too large");
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
    const int64_t K = p->K;
    ProfScope ps("slos_encode_gemm", 0.0, s);
    dim3 grid((unsigned)((K + kGT - 1) / kGT), (unsigned)((batch + kGT - 1) / kGT));
    encode_gemm_kernel<<<grid, dim3(16, 16), 0, s>>>(reinterpret_cast<const float2 *>(X), buf[0], p->tab.gfact, batch,
                                                     K, output == SLOS_OUT_PROBS, out);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return fail(SLOS_ERR_CUDA, std::string("slos_encoded_forward: ") + cudaGetErrorString(e));
    return SLOS_OK;
}

}  // extern "C"
