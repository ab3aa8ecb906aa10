// Shot sampling from output distributions (the hardware-aware design
// section: MerlinProcessor returns counts of a finite number of shots).
//
// Exact integer inversion of the cumulative distribution: weights are fixed
// point, P(t) = floor(p(t) 2^32); C(t) = P(0) + ... + P(t) and the total T are
// exact 64-bit integers (K < 2^31 weights below 2^32 + 1 each), so no
// summation order can change a decision.  A draw u in [0, 1) becomes the
// target floor(floor(u 2^32) T / 2^32) (a 96-bit product) and the outcome is
// the first t with C(t) > target.  Three kernels: per-chunk sums of 256
// weights, an in-place inclusive scan of the chunk sums per instance, and one
// thread per shot that binary-searches the chunk prefix and walks the chunk.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/slos.h"
#include "plan.h"
#include "profile.h"

namespace slos {
slos_status_t fail(slos_status_t st, const std::string &msg);

constexpr int kSampleChunk = 256;
constexpr int kScanThreads = 1024;

__device__ __forceinline__ uint64_t fixed32(float x) {
    return x > 0.f ? __float2ull_rz(x * 4294967296.0f) : 0ull;  // NaN and negatives weigh nothing
}

__global__ void __launch_bounds__(kSampleChunk) chunk_sum_kernel(const float *p, int64_t K, int64_t nchunks,
                                                                 uint64_t *sums) {
    __shared__ uint64_t red[kSampleChunk / 32];
    const int b = blockIdx.y;
    const int64_t c = (int64_t)blockIdx.x * kSampleChunk + threadIdx.x;
    uint64_t v = c < K ? fixed32(p[(size_t)b * K + c]) : 0ull;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t s = 0;
        for (int w = 0; w < kSampleChunk / 32; ++w) s += red[w];
        sums[(size_t)b * nchunks + blockIdx.x] = s;
    }
}

// inclusive scan of one instance's chunk sums, in place: each thread takes a
// contiguous segment, the segment totals are scanned in shared memory
__global__ void __launch_bounds__(kScanThreads) chunk_scan_kernel(uint64_t *sums, int64_t nchunks) {
    __shared__ uint64_t seg[kScanThreads];
    uint64_t *row = sums + (size_t)blockIdx.x * nchunks;
    const int64_t per = (nchunks + kScanThreads - 1) / kScanThreads;
    const int64_t lo = threadIdx.x * per, hi = min(lo + per, nchunks);
    uint64_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += row[i];
    seg[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < kScanThreads; off <<= 1) {
        const uint64_t add = threadIdx.x >= off ? seg[threadIdx.x - off] : 0ull;
        __syncthreads();
        seg[threadIdx.x] += add;
        __syncthreads();
    }
    uint64_t run = threadIdx.x > 0 ? seg[threadIdx.x - 1] : 0ull;
    for (int64_t i = lo; i < hi; ++i) {
        run += row[i];
        row[i] = run;
    }
}

__global__ void sample_kernel(const float *p, int64_t K, int64_t nchunks, const uint64_t *prefix, const float *u,
                              int B, int shots, int32_t *samples, int32_t *counts) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)B * shots) return;
    const int b = (int)(idx / shots);
    const uint64_t *pre = prefix + (size_t)b * nchunks;
    const uint64_t T = pre[nchunks - 1];
    if (T == 0) {
        samples[idx] = -1;  // no outcome carries any weight
        return;
    }
    const float x = u[idx];
    const uint64_t U32 = x > 0.f ? (uint64_t)__float2uint_rz(x * 4294967296.0f) : 0ull;  // saturates at 2^32 - 1
    const uint64_t lo64 = T * U32, hi64 = __umul64hi(T, U32);
    const uint64_t target = (hi64 << 32) | (lo64 >> 32);  // floor(U32 T / 2^32)
    // first chunk whose inclusive prefix exceeds the target
    int64_t l = 0, h = nchunks - 1;
    while (l < h) {
        const int64_t mid = (l + h) >> 1;
        if (pre[mid] > target) h = mid;
        else l = mid + 1;
    }
    uint64_t acc = l > 0 ? pre[l - 1] : 0ull;
    const float *pb = p + (size_t)b * K;
    const int64_t end = min((l + 1) * (int64_t)kSampleChunk, K);
    int64_t t = l * kSampleChunk;
    for (; t < end; ++t) {
        acc += fixed32(pb[t]);
        if (acc > target) break;
    }
    if (t >= end) t = end - 1;  // unreachable: the chunk's prefix exceeds the target
    samples[idx] = (int32_t)t;
    if (counts) atomicAdd(counts + (size_t)b * K + t, 1);
}

static int64_t chunks_of(const slos_plan_s *p) { return (p->K + kSampleChunk - 1) / kSampleChunk; }

}  // namespace slos

using namespace slos;

extern "C" {

slos_status_t slos_sample_workspace_bytes(slos_plan_t p, int batch, size_t *bytes) {
    if (!p || p->kind != 0 || !bytes) return fail(SLOS_ERR_INVALID_ARG, "slos_sample_workspace_bytes: bad argument");
    if (batch < 0) return fail(SLOS_ERR_INVALID_ARG, "slos_sample_workspace_bytes: negative batch");
    *bytes = (size_t)batch * chunks_of(p) * sizeof(uint64_t);
    return SLOS_OK;
}

slos_status_t slos_sample(slos_plan_t p, const float *probs, int batch, int shots, const float *uniforms,
                          int32_t *samples, int32_t *counts, void *workspace, size_t workspace_bytes, void *stream) {
    if (!p || p->kind != 0) return fail(SLOS_ERR_INVALID_ARG, "slos_sample: not a single-shape plan");
    if (batch < 0 || shots < 0) return fail(SLOS_ERR_INVALID_ARG, "slos_sample: negative batch or shots");
    if (batch > 65535) return fail(SLOS_ERR_UNSUPPORTED, "slos_sample: at most 65535 instances per call");
    if (batch == 0) return SLOS_OK;
    if (!probs || (shots > 0 && (!uniforms || !samples)))
        return fail(SLOS_ERR_INVALID_ARG, "slos_sample: NULL pointer");
    const int64_t nch = chunks_of(p);
    if (!workspace || workspace_bytes < (size_t)batch * nch * sizeof(uint64_t))
        return fail(SLOS_ERR_INVALID_ARG, "slos_sample: workspace too small (slos_sample_workspace_bytes)");
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t *pre = reinterpret_cast<uint64_t *>(workspace);
    ProfScope ps("slos_sample", (double)batch * (4.0 * p->K) + (double)batch * shots * 8.0, s);
    cudaError_t e;
    if (counts && (e = cudaMemsetAsync(counts, 0, (size_t)batch * p->K * sizeof(int32_t), s)) != cudaSuccess)
        return fail(SLOS_ERR_CUDA, std::string("slos_sample: ") + cudaGetErrorString(e));
    chunk_sum_kernel<<<dim3((unsigned)nch, batch), kSampleChunk, 0, s>>>(probs, p->K, nch, pre);
    chunk_scan_kernel<<<batch, kScanThreads, 0, s>>>(pre, nch);
    const int64_t total = (int64_t)batch * shots;
    if (total > 0)
        sample_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(probs, p->K, nch, pre, uniforms, batch, shots,
                                                                      samples, counts);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return fail(SLOS_ERR_CUDA, std::string("slos_sample: ") + cudaGetErrorString(e));
    return SLOS_OK;
}

}  // extern "C"
