// Measurement strategies on top of an output distribution (Sec. II-A.3,
// QuantumLayer: per-mode photon-number expectations) and renormalisation onto
// the plan's space, each with its backward.  Caller buffers only; one CTA per
// instance for the reductions, summed in a fixed order (warp shuffles, then
// the warps in index order) so that every value is reproducible.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/slos.h"
#include "common.cuh"
#include "dfloat.cuh"
#include "plan.h"
#include "profile.h"

namespace slos {
slos_status_t fail(slos_status_t st, const std::string &msg);

constexpr int kMeasThreads = 256;
constexpr int kMeasWarps = kMeasThreads / 32;

// out[b][j] = sum_t occ[t][j] p[b][t]
__global__ void __launch_bounds__(kMeasThreads) expect_fwd_kernel(const float *p, const uint8_t *occ, int64_t K, int m,
                                                                  float *out) {
    __shared__ float red[kMeasWarps][kMaxModes];
    const int b = blockIdx.x;
    const float *pb = p + (size_t)b * K;
    float acc[kMaxModes];
#pragma unroll
    for (int j = 0; j < kMaxModes; ++j) acc[j] = 0.f;
    for (int64_t c = threadIdx.x; c < K; c += kMeasThreads) {
        const float v = pb[c];
        const uint8_t *row = occ + (size_t)c * m;
#pragma unroll
        for (int j = 0; j < kMaxModes; ++j)
            if (j < m) acc[j] += (float)__ldg(row + j) * v;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kMaxModes; ++j) {
        float v = acc[j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][j] = v;
    }
    __syncthreads();
    if (threadIdx.x < m) {
        float v = 0.f;
        for (int w = 0; w < kMeasWarps; ++w) v += red[w][threadIdx.x];
        out[(size_t)b * m + threadIdx.x] = v;
    }
}

// dp[b][t] = sum_j occ[t][j] dout[b][j]
__global__ void __launch_bounds__(kMeasThreads) expect_bwd_kernel(const float *dout, const uint8_t *occ, int64_t K,
                                                                  int m, float *dp) {
    __shared__ float d[kMaxModes];
    const int b = blockIdx.y;
    if (threadIdx.x < m) d[threadIdx.x] = dout[(size_t)b * m + threadIdx.x];
    __syncthreads();
    const int64_t c = (int64_t)blockIdx.x * kMeasThreads + threadIdx.x;
    if (c >= K) return;
    const uint8_t *row = occ + (size_t)c * m;
    float v = 0.f;
    for (int j = 0; j < m; ++j) v += (float)__ldg(row + j) * d[j];
    dp[(size_t)b * K + c] = v;
}

// block sum of one double-float per thread, fixed order; every thread gets it
__device__ dfl block_sum(dfl v, dfl *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        const dfl w = {__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
        v = df_add(v, w);
    }
    if (lane == 0) red[warp] = v;
    __syncthreads();
    dfl s = df_zero();
    for (int w = 0; w < kMeasWarps; ++w) s = df_add(s, red[w]);
    __syncthreads();
    return s;
}

// Z = sum_t p[t]; q[t] = p[t] / Z  (sums in double-float, dfloat.cuh)
__global__ void __launch_bounds__(kMeasThreads) renorm_fwd_kernel(const float *p, int64_t K, float *q, float *Z) {
    __shared__ dfl red[kMeasWarps];
    const int b = blockIdx.x;
    const float *pb = p + (size_t)b * K;
    dfl acc = df_zero();
    for (int64_t c = threadIdx.x; c < K; c += kMeasThreads) acc = df_add_f(acc, pb[c]);
    const float z = df_float(block_sum(acc, red));
    const float inv = z > 0.f ? 1.f / z : 0.f;
    float *qb = q + (size_t)b * K;
    for (int64_t c = threadIdx.x; c < K; c += kMeasThreads) qb[c] = pb[c] * inv;
    if (threadIdx.x == 0) Z[b] = z;
}

// dp[t] = (dq[t] - sum_s dq[s] q[s]) / Z
__global__ void __launch_bounds__(kMeasThreads) renorm_bwd_kernel(const float *q, const float *Z, const float *dq,
                                                                  int64_t K, float *dp) {
    __shared__ dfl red[kMeasWarps];
    const int b = blockIdx.x;
    const float *qb = q + (size_t)b * K, *dqb = dq + (size_t)b * K;
    dfl acc = df_zero();
    for (int64_t c = threadIdx.x; c < K; c += kMeasThreads) acc = df_add(acc, two_prod(dqb[c], qb[c]));
    const float sdot = df_float(block_sum(acc, red));
    const float z = Z[b];
    const float inv = z > 0.f ? 1.f / z : 0.f;
    float *dpb = dp + (size_t)b * K;
    for (int64_t c = threadIdx.x; c < K; c += kMeasThreads) dpb[c] = (dqb[c] - sdot) * inv;
}

static slos_status_t check(slos_plan_t p, int batch, const char *who) {
    if (!p || p->kind != 0) return fail(SLOS_ERR_INVALID_ARG, std::string(who) + ": not a single-shape plan");
    if (batch < 0) return fail(SLOS_ERR_INVALID_ARG, std::string(who) + ": negative batch");
    if (batch > 65535) return fail(SLOS_ERR_UNSUPPORTED, std::string(who) + ": at most 65535 instances per call");
    return SLOS_OK;
}

static slos_status_t launched(const char *who) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(SLOS_ERR_CUDA, std::string(who) + ": " + cudaGetErrorString(e));
    return SLOS_OK;
}

}  // namespace slos

using namespace slos;

extern "C" {

slos_status_t slos_expectations(slos_plan_t p, const float *probs, int batch, float *out, void *stream) {
    slos_status_t st = check(p, batch, "slos_expectations");
    if (st != SLOS_OK) return st;
    if (!p->tab.occ) return fail(SLOS_ERR_UNSUPPORTED, "slos_expectations: plan too large for its occupation table");
    if (batch == 0) return SLOS_OK;
    if (!probs || !out) return fail(SLOS_ERR_INVALID_ARG, "slos_expectations: NULL pointer");
    cudaStream_t s = (cudaStream_t)stream;
    ProfScope ps("slos_expectations", (double)batch * (4.0 * p->K + 4.0 * p->m), s);
    expect_fwd_kernel<<<batch, kMeasThreads, 0, s>>>(probs, p->tab.occ, p->K, p->m, out);
    return launched("slos_expectations");
}

slos_status_t slos_expectations_backward(slos_plan_t p, const float *dout, int batch, float *dprobs, void *stream) {
    slos_status_t st = check(p, batch, "slos_expectations_backward");
    if (st != SLOS_OK) return st;
    if (!p->tab.occ)
        return fail(SLOS_ERR_UNSUPPORTED, "slos_expectations_backward: plan too large for its occupation table");
    if (batch == 0) return SLOS_OK;
    if (!dout || !dprobs) return fail(SLOS_ERR_INVALID_ARG, "slos_expectations_backward: NULL pointer");
    cudaStream_t s = (cudaStream_t)stream;
    ProfScope ps("slos_expectations_bwd", (double)batch * (4.0 * p->K + 4.0 * p->m), s);
    dim3 grid((unsigned)((p->K + kMeasThreads - 1) / kMeasThreads), batch);
    expect_bwd_kernel<<<grid, kMeasThreads, 0, s>>>(dout, p->tab.occ, p->K, p->m, dprobs);
    return launched("slos_expectations_backward");
}

slos_status_t slos_renormalise(slos_plan_t p, const float *pr, int batch, float *q, float *Z, void *stream) {
    slos_status_t st = check(p, batch, "slos_renormalise");
    if (st != SLOS_OK) return st;
    if (batch == 0) return SLOS_OK;
    if (!pr || !q || !Z) return fail(SLOS_ERR_INVALID_ARG, "slos_renormalise: NULL pointer");
    cudaStream_t s = (cudaStream_t)stream;
    ProfScope ps("slos_renormalise", (double)batch * 8.0 * p->K, s);
    renorm_fwd_kernel<<<batch, kMeasThreads, 0, s>>>(pr, p->K, q, Z);
    return launched("slos_renormalise");
}

slos_status_t slos_renormalise_backward(slos_plan_t p, const float *q, const float *Z, const float *dq, int batch,
                                        float *dp, void *stream) {
    slos_status_t st = check(p, batch, "slos_renormalise_backward");
    if (st != SLOS_OK) return st;
    if (batch == 0) return SLOS_OK;
    if (!q || !Z || !dq || !dp) return fail(SLOS_ERR_INVALID_ARG, "slos_renormalise_backward: NULL pointer");
    cudaStream_t s = (cudaStream_t)stream;
    ProfScope ps("slos_renormalise_bwd", (double)batch * 12.0 * p->K, s);
    renorm_bwd_kernel<<<batch, kMeasThreads, 0, s>>>(q, Z, dq, p->K, dp);
    return launched("slos_renormalise_backward");
}

}  // extern "C"
