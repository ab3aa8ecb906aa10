// Learned surrogate of the m=12, n=6 layer: a BF16 MLP, phases -> log output
// distribution, trained on distributions produced by the exact SLOS path.
//
//   features  x = [sin phi, cos phi]            (2 * n_phases)
//   hidden    h_l = GELU(h_{l-1} W_l^T + b_l)   (n_hidden layers of width H)
//   logits    z = h_L W_out^T + b_out           (K outputs), q = softmax(z)
//   loss      KL(p || q) = sum_t p_t (log p_t - log q_t),  dL/dz = q - p
//
// Every matrix product runs on the tcgen05 GEMM (tc_gemm.cuh); weights are
// kept as FP32 masters plus BF16 copies W [out][in] (forward) and W^T
// [in][out] (input gradient), refreshed by the Adam kernel.  Weight
// gradients need the batch as the reduction (K-major) axis, so activations
// and output gradients are transposed into [features][batch] first.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdio>
#include <cstring>
#include <cudaTypedefs.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <random>
#include <string>
#include <vector>

#include "../../include/surrogate.h"
#include "profile.h"
#include "tc_gemm.cuh"

namespace slos {
slos_status_t fail(slos_status_t st, const std::string &msg);
}

using namespace slos;
using namespace slos::tc;

namespace {

__device__ int g_tc_err = 0;

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// K-major BF16 matrix [rows][cols] (row stride ld elements), box 64 x box_rows.
bool make_map(CUtensorMap *map, const void *ptr, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int *err_ptr() {
    static int *p = nullptr;
    if (!p) cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_tc_err);
    return p;
}

bool g_attr_done[64] = {false};
int g_sm_count[64] = {0};

int sm_count() {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 148;
    if (g_sm_count[dev] <= 0) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        g_sm_count[dev] = n > 0 ? n : 148;
    }
    return g_sm_count[dev];
}

template <int EPI>
cudaError_t set_attr() {
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(tc_gemm_persist_kernel<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
}

cudaError_t init_attrs() {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && g_attr_done[dev]) return cudaSuccess;
    cudaError_t e;
    if ((e = set_attr<TC_F32>()) != cudaSuccess) return e;
    if ((e = set_attr<TC_F32_BIAS>()) != cudaSuccess) return e;
    if ((e = set_attr<TC_GELU>()) != cudaSuccess) return e;
    if ((e = set_attr<TC_GELU_BWD>()) != cudaSuccess) return e;
    if ((e = set_attr<TC_F32_ACCUM>()) != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) g_attr_done[dev] = true;
    return cudaSuccess;
}

// C[M][N] = A[M][K] . B[N][K]^T with epilogue EPI.  lda/ldb in elements.
slos_status_t gemm(int epi, int M, int N, int K, const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *Bm,
                   int64_t ldb, void *C, int ldc, const float *bias, __nv_bfloat16 *aux, cudaStream_t s) {
    if (M <= 0 || N <= 0 || K <= 0) return SLOS_OK;
    if ((K % 8) || (lda % 8) || (ldb % 8) || (reinterpret_cast<uintptr_t>(A) & 15) ||
        (reinterpret_cast<uintptr_t>(Bm) & 15))
        return fail(SLOS_ERR_INVALID_ARG, "tensor-core GEMM: K, row strides must be multiples of 8 elements and "
                                          "operands 16-byte aligned");
    cudaError_t e = init_attrs();
    if (e != cudaSuccess) return fail(SLOS_ERR_CUDA, std::string("GEMM attributes: ") + cudaGetErrorString(e));
    CUtensorMap ta, tb;
    if (!make_map(&ta, A, M, K, lda, BM) || !make_map(&tb, Bm, N, K, ldb, BN))
        return fail(SLOS_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    TcArgs g;
    g.M = M;
    g.N = N;
    g.K = K;
    g.C = C;
    g.ldc = ldc;
    g.bias = bias;
    g.aux = aux;
    g.err = err_ptr();
    g.colscale = nullptr;
    g.amps = 0;
    // persistent CTAs, one per SM (the shared-memory ring allows no second)
    const int64_t tiles = (int64_t)((N + BN - 1) / BN) * ((M + BM - 1) / BM);
    const unsigned grid = (unsigned)std::min<int64_t>(tiles, sm_count());
    ProfScope ps("tc_gemm", 2.0 * M * N * K, s);  // flops, not bytes
    constexpr int T = kPersistThreads;
    switch (epi) {
        case TC_F32: tc_gemm_persist_kernel<TC_F32><<<grid, T, SMEM_BYTES, s>>>(ta, tb, g); break;
        case TC_F32_BIAS: tc_gemm_persist_kernel<TC_F32_BIAS><<<grid, T, SMEM_BYTES, s>>>(ta, tb, g); break;
        case TC_GELU: tc_gemm_persist_kernel<TC_GELU><<<grid, T, SMEM_BYTES, s>>>(ta, tb, g); break;
        case TC_GELU_BWD: tc_gemm_persist_kernel<TC_GELU_BWD><<<grid, T, SMEM_BYTES, s>>>(ta, tb, g); break;
        case TC_F32_ACCUM: tc_gemm_persist_kernel<TC_F32_ACCUM><<<grid, T, SMEM_BYTES, s>>>(ta, tb, g); break;
        default: return fail(SLOS_ERR_INVALID_ARG, "GEMM epilogue");
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(SLOS_ERR_CUDA, std::string("GEMM launch: ") + cudaGetErrorString(e));
    return SLOS_OK;
}

// ---------------------------------------------------------------- small kernels
// phase j of row b: in[b][j], or with H > 0 harmonics of nx inputs per row,
// (j / nx + 1) * in[b][j % nx]
__global__ void features_kernel(const float *in, int B, int P, int H, int nx, __nv_bfloat16 *x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)B * P) return;
    const int64_t b = i / P, j = i % P;
    const float phi = H > 0 ? (float)(j / nx + 1) * in[b * nx + j % nx] : in[i];
    float s, c;
    sincosf(phi, &s, &c);
    x[b * 2 * P + j] = __float2bfloat16(s);
    x[b * 2 * P + P + j] = __float2bfloat16(c);
}

// out[c][r] = in[r][c] for a [R][C] bf16 matrix (32 x 32 tiles through shared memory)
__global__ void transpose_kernel(const __nv_bfloat16 *in, int R, int C, __nv_bfloat16 *out) {
    __shared__ __nv_bfloat16 t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        if (r < R && c < C) t[i][threadIdx.x] = in[(int64_t)r * C + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (r < R && c < C) out[(int64_t)c * R + r] = t[threadIdx.x][i];
    }
}

// One block per row: q = softmax(z); loss_row = sum p (log p - log q);
// dz = (q - p) * scale (bf16); optionally q out (float).
__global__ void softmax_kl_kernel(const float *z, const float *p, int K, float scale, __nv_bfloat16 *dz,
                                  float *loss_rows, float *q_out) {
    const int64_t r = blockIdx.x;
    const float *zr = z + r * K;
    __shared__ float red[32];
    float mx = -INFINITY;
    for (int i = threadIdx.x; i < K; i += blockDim.x) mx = fmaxf(mx, zr[i]);
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : -INFINITY;
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) red[0] = v;
    }
    __syncthreads();
    mx = red[0];
    __syncthreads();
    float se = 0.f;
    for (int i = threadIdx.x; i < K; i += blockDim.x) se += expf(zr[i] - mx);
    for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = se;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) red[0] = v;
    }
    __syncthreads();
    const float lse = mx + logf(red[0]);
    __syncthreads();
    float kl = 0.f;
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
        const float lq = zr[i] - lse;
        const float q = expf(lq);
        const float pi = p ? p[r * K + i] : 0.f;
        if (pi > 0.f) kl += pi * (logf(pi) - lq);
        if (dz) dz[r * K + i] = __float2bfloat16((q - pi) * scale);
        if (q_out) q_out[r * K + i] = q;
    }
    for (int o = 16; o > 0; o >>= 1) kl += __shfl_xor_sync(0xffffffffu, kl, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = kl;
    __syncthreads();
    if (threadIdx.x == 0) {
        float v = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
        if (loss_rows) loss_rows[r] = v;
    }
}

// db[n] = sum_r d[r][n] (bf16 in, float out), in row order
__global__ void colsum_kernel(const __nv_bfloat16 *d, int R, int N, float *db) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int r = 0; r < R; ++r) s += __bfloat162float(d[(int64_t)r * N + n]);
    db[n] = s;
}

struct AdamArgs {
    float *w, *m, *v;
    const float *g;
    __nv_bfloat16 *wb, *wbt;  // [out][in], [in][out] (may be null)
    int64_t n;
    int rows, cols;           // for the transposed copy
    float lr, b1, b2, eps, c1, c2;  // c1 = 1/(1-b1^t), c2 = 1/(1-b2^t)
};

__global__ void adam_kernel(AdamArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const float g = a.g[i];
    const float m = a.b1 * a.m[i] + (1.f - a.b1) * g;
    const float v = a.b2 * a.v[i] + (1.f - a.b2) * g * g;
    a.m[i] = m;
    a.v[i] = v;
    const float w = a.w[i] - a.lr * (m * a.c1) / (sqrtf(v * a.c2) + a.eps);
    a.w[i] = w;
    const __nv_bfloat16 wb = __float2bfloat16(w);
    if (a.wb) a.wb[i] = wb;
    if (a.wbt) {
        const int64_t r = i / a.cols, c = i % a.cols;
        a.wbt[c * a.rows + r] = wb;
    }
}



// ---------------------------------------------------------------- checks
// tv[i] = 1/2 sum_t |q[rows[i]][t] - p[i][t]|   (one block per checked row)
__global__ void tv_rows_kernel(const float *q, const int *rows, const float *p, int K, float *tv) {
    const int i = blockIdx.x;
    const float *qr = q + (int64_t)rows[i] * K;
    const float *pr = p + (int64_t)i * K;
    float s = 0.f;
    for (int t = threadIdx.x; t < K; t += blockDim.x) s += fabsf(qr[t] - pr[t]);
    __shared__ float red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float v = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
        tv[i] = 0.5f * v;
    }
}

// marg[b][j] = sum_t q[b][t] * occ[t][j]    (one block per row)
__global__ void marginals_kernel(const float *q, int K, const uint8_t *occ, int m, float *marg) {
    const int b = blockIdx.x;
    __shared__ float acc[32][33];
    float loc[32];
    for (int j = 0; j < 32; ++j) loc[j] = 0.f;
    const float *qr = q + (int64_t)b * K;
    for (int t = threadIdx.x; t < K; t += blockDim.x) {
        const float v = qr[t];
        for (int j = 0; j < m; ++j) loc[j] += v * (float)occ[(int64_t)t * m + j];
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int j = 0; j < m; ++j) {
        float v = loc[j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (l == 0) acc[w][j] = v;
    }
    __syncthreads();
    if (threadIdx.x < m) {
        float v = 0.f;
        for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) v += acc[ww][threadIdx.x];
        marg[(int64_t)b * m + threadIdx.x] = v;
    }
}

// exact mean photon numbers <n_j> = sum_i |U[b][j][i]|^2 s_i; flag[b] = 1 if
// max_j |marg[b][j] - <n_j>| > tol (flag is OR-ed, never cleared here)
struct ScreenArgs {
    const float2 *U;
    const float *marg;
    int B, m;
    float s[24];
    float tol;
    int *flag;
};
__global__ void screen_kernel(ScreenArgs a) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= a.B) return;
    // sum over modes of |exact <n_j> - surrogate <n_j>|: with the sign
    // pattern w_j = +-1 of those differences, f(t) = sum_j w_j t_j lies in
    // [-n, n] and the differences sum to zero, so sum_j |d_j| =
    // sum_t f(t) (p_t - q_t) <= 2 n TV(p, q): a sum above 2 n tol proves TV > tol
    float l1 = 0.f;
    for (int j = 0; j < a.m; ++j) {
        float nj = 0.f;
        for (int i = 0; i < a.m; ++i) {
            const float2 u = a.U[((int64_t)b * a.m + j) * a.m + i];
            nj += (u.x * u.x + u.y * u.y) * a.s[i];
        }
        l1 += fabsf(nj - a.marg[(int64_t)b * a.m + j]);
    }
    if (l1 > a.tol) a.flag[b] = 1;
}

// dst[rows[i]] = src[i] (K floats per row)
__global__ void scatter_rows_kernel(const float *src, const int *rows, int K, float *dst) {
    const int i = blockIdx.x;
    const float *sr = src + (int64_t)i * K;
    float *dr = dst + (int64_t)rows[i] * K;
    for (int t = threadIdx.x; t < K; t += blockDim.x) dr[t] = sr[t];
}
// dst[i] = src[rows[i]] (n_phases floats per row)
__global__ void gather_rows_kernel(const float *src, const int *rows, int W, float *dst) {
    const int i = blockIdx.x;
    for (int t = threadIdx.x; t < W; t += blockDim.x) dst[(int64_t)i * W + t] = src[(int64_t)rows[i] * W + t];
}

}  // namespace

// ======================================================================== model
struct surr_model_s {
    int n_phases, in_dim, hidden, n_layers, K, max_batch;
    int harmonics = 0;  // > 0: inputs are n_phases / harmonics values x, phases h x for h = 1..harmonics
    // parameters: layer l = 0..n_layers (last = output layer)
    std::vector<int> fan_in, fan_out;
    std::vector<float *> w, b, mw, vw, mb, vb, gw, gb;
    std::vector<__nv_bfloat16 *> wb, wbt;
    // activations
    __nv_bfloat16 *x0 = nullptr;                 // [B][in_dim]
    std::vector<__nv_bfloat16 *> z, h;           // [n_layers][B][H]
    float *logits = nullptr;                     // [B][K]
    __nv_bfloat16 *dlog = nullptr;               // [B][K]
    __nv_bfloat16 *dh[2] = {nullptr, nullptr};   // [B][H] ping-pong
    __nv_bfloat16 *tA = nullptr, *tB = nullptr;  // transposes: [max(K,H)][B], [max(H,in)][B]
    float *loss_rows = nullptr;                  // [B]
    int step = 0;
    float lr = 1e-3f;
};

namespace {

slos_status_t cuda_alloc(void **p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) return fail(SLOS_ERR_OOM, "surrogate: device allocation failed");
    return SLOS_OK;
}

slos_status_t launch_check(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(SLOS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return SLOS_OK;
}

slos_status_t transpose(const __nv_bfloat16 *in, int R, int C, __nv_bfloat16 *out, cudaStream_t s) {
    dim3 grid((C + 31) / 32, (R + 31) / 32), block(32, 8);
    ProfScope ps("surr_transpose", 4.0 * R * C, s);
    transpose_kernel<<<grid, block, 0, s>>>(in, R, C, out);
    return launch_check("transpose");
}

}  // namespace

extern "C" {

slos_status_t surr_gemm_bf16(int epi, int M, int N, int K, const void *A, int64_t lda, const void *B, int64_t ldb,
                             void *C, int ldc, const float *bias, void *aux, void *stream) {
    return gemm(epi, M, N, K, reinterpret_cast<const __nv_bfloat16 *>(A), lda, reinterpret_cast<const __nv_bfloat16 *>(B),
                ldb, C, ldc, bias, reinterpret_cast<__nv_bfloat16 *>(aux), (cudaStream_t)stream);
}

slos_status_t surr_sync_status(void *stream) {
    int h = 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(SLOS_ERR_CUDA, "surr_sync_status: stream error");
    if (cudaMemcpyFromSymbol(&h, g_tc_err, sizeof(int)) != cudaSuccess)
        return fail(SLOS_ERR_CUDA, "surr_sync_status: read error word");
    if (h != 0) {
        int z = 0;
        cudaMemcpyToSymbol(g_tc_err, &z, sizeof(int));
        return fail(SLOS_ERR_TIMEOUT, "tensor-core GEMM: a bounded pipeline wait ran out (code " + std::to_string(h) + ")");
    }
    return SLOS_OK;
}

slos_status_t surr_create(int n_phases, int hidden, int n_hidden_layers, int n_outputs, int max_batch,
                          unsigned long long seed, surr_model_t *out) {
    if (!out) return fail(SLOS_ERR_INVALID_ARG, "surr_create: NULL out");
    *out = nullptr;
    if (n_phases <= 0 || hidden <= 0 || n_hidden_layers <= 0 || n_outputs <= 0 || max_batch <= 0 ||
        (2 * n_phases) % 8 || hidden % 8 || n_outputs % 8 || max_batch % 8)
        return fail(SLOS_ERR_INVALID_ARG, "surr_create: sizes must be positive; 2*n_phases, hidden, n_outputs and "
                                          "max_batch multiples of 8");
    surr_model_s *M = new surr_model_s();
    M->n_phases = n_phases;
    M->in_dim = 2 * n_phases;
    M->hidden = hidden;
    M->n_layers = n_hidden_layers;
    M->K = n_outputs;
    M->max_batch = max_batch;
    std::mt19937_64 rng(seed);
    const int L = n_hidden_layers + 1;
    for (int l = 0; l < L; ++l) {
        const int fi = l == 0 ? M->in_dim : hidden;
        const int fo = l == L - 1 ? n_outputs : hidden;
        M->fan_in.push_back(fi);
        M->fan_out.push_back(fo);
        const size_t nw = (size_t)fi * fo;
        float *w, *b, *mw, *vw, *mb, *vb, *gw, *gb;
        __nv_bfloat16 *wb, *wbt;
        slos_status_t st;
        if ((st = cuda_alloc((void **)&w, nw * 4)) || (st = cuda_alloc((void **)&mw, nw * 4)) ||
            (st = cuda_alloc((void **)&vw, nw * 4)) || (st = cuda_alloc((void **)&gw, nw * 4)) ||
            (st = cuda_alloc((void **)&b, fo * 4)) || (st = cuda_alloc((void **)&mb, fo * 4)) ||
            (st = cuda_alloc((void **)&vb, fo * 4)) || (st = cuda_alloc((void **)&gb, fo * 4)) ||
            (st = cuda_alloc((void **)&wb, nw * 2)) || (st = cuda_alloc((void **)&wbt, nw * 2))) {
            surr_destroy(M);
            return st;
        }
        // He-uniform init on the host (seeded), zero bias and moments
        std::vector<float> hw(nw);
        const float a = std::sqrt(6.0f / fi) * (l == L - 1 ? 0.5f : 1.0f);
        std::uniform_real_distribution<float> U(-a, a);
        for (auto &x : hw) x = U(rng);
        cudaMemcpy(w, hw.data(), nw * 4, cudaMemcpyHostToDevice);
        cudaMemset(b, 0, fo * 4);
        cudaMemset(mw, 0, nw * 4);
        cudaMemset(vw, 0, nw * 4);
        cudaMemset(mb, 0, fo * 4);
        cudaMemset(vb, 0, fo * 4);
        M->w.push_back(w);
        M->b.push_back(b);
        M->mw.push_back(mw);
        M->vw.push_back(vw);
        M->mb.push_back(mb);
        M->vb.push_back(vb);
        M->gw.push_back(gw);
        M->gb.push_back(gb);
        M->wb.push_back(wb);
        M->wbt.push_back(wbt);
        // bf16 copies
        AdamArgs aa;
        memset(&aa, 0, sizeof(aa));
        std::vector<__nv_bfloat16> hb(nw), hbt(nw);
        for (size_t i = 0; i < nw; ++i) {
            hb[i] = __float2bfloat16(hw[i]);
            const size_t r = i / fi, c = i % fi;
            hbt[c * fo + r] = hb[i];
        }
        cudaMemcpy(wb, hb.data(), nw * 2, cudaMemcpyHostToDevice);
        cudaMemcpy(wbt, hbt.data(), nw * 2, cudaMemcpyHostToDevice);
    }
    const size_t B = max_batch;
    const size_t big = std::max<size_t>(std::max(n_outputs, hidden), M->in_dim);
    slos_status_t st;
    if ((st = cuda_alloc((void **)&M->x0, B * M->in_dim * 2)) || (st = cuda_alloc((void **)&M->logits, B * n_outputs * 4)) ||
        (st = cuda_alloc((void **)&M->dlog, B * n_outputs * 2)) || (st = cuda_alloc((void **)&M->dh[0], B * hidden * 2)) ||
        (st = cuda_alloc((void **)&M->dh[1], B * hidden * 2)) || (st = cuda_alloc((void **)&M->tA, big * B * 2)) ||
        (st = cuda_alloc((void **)&M->tB, big * B * 2)) || (st = cuda_alloc((void **)&M->loss_rows, B * 4))) {
        surr_destroy(M);
        return st;
    }
    for (int l = 0; l < n_hidden_layers; ++l) {
        __nv_bfloat16 *z, *h;
        if ((st = cuda_alloc((void **)&z, B * hidden * 2)) || (st = cuda_alloc((void **)&h, B * hidden * 2))) {
            surr_destroy(M);
            return st;
        }
        M->z.push_back(z);
        M->h.push_back(h);
    }
    *out = M;
    return SLOS_OK;
}

slos_status_t surr_destroy(surr_model_t M) {
    if (!M) return SLOS_OK;
    for (auto v : {&M->w, &M->b, &M->mw, &M->vw, &M->mb, &M->vb, &M->gw, &M->gb})
        for (float *p : *v) cudaFree(p);
    for (auto p : M->wb) cudaFree(p);
    for (auto p : M->wbt) cudaFree(p);
    for (auto p : M->z) cudaFree(p);
    for (auto p : M->h) cudaFree(p);
    cudaFree(M->x0);
    cudaFree(M->logits);
    cudaFree(M->dlog);
    cudaFree(M->dh[0]);
    cudaFree(M->dh[1]);
    cudaFree(M->tA);
    cudaFree(M->tB);
    cudaFree(M->loss_rows);
    delete M;
    return SLOS_OK;
}

slos_status_t surr_set_input_harmonics(surr_model_t M, int harmonics) {
    if (!M) return fail(SLOS_ERR_INVALID_ARG, "surr_set_input_harmonics: NULL model");
    if (harmonics < 0 || (harmonics > 0 && M->n_phases % harmonics))
        return fail(SLOS_ERR_INVALID_ARG, "surr_set_input_harmonics: harmonics must divide n_phases");
    M->harmonics = harmonics;
    return SLOS_OK;
}

static slos_status_t forward_impl(surr_model_t M, const float *phases, int B, cudaStream_t s) {
    if (B <= 0 || B > M->max_batch || B % 8) return fail(SLOS_ERR_INVALID_ARG, "surrogate: batch must be in (0, max_batch], multiple of 8");
    const int64_t n = (int64_t)B * M->n_phases;
    {
        ProfScope ps("surr_features", 4.0 * n + 4.0 * n, s);
        features_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
            phases, B, M->n_phases, M->harmonics, M->harmonics > 0 ? M->n_phases / M->harmonics : M->n_phases, M->x0);
    }
    slos_status_t st = launch_check("features");
    if (st) return st;
    const __nv_bfloat16 *x = M->x0;
    int xd = M->in_dim;
    for (int l = 0; l < M->n_layers; ++l) {
        st = gemm(TC_GELU, B, M->hidden, xd, x, xd, M->wb[l], xd, M->h[l], M->hidden, M->b[l], M->z[l], s);
        if (st) return st;
        x = M->h[l];
        xd = M->hidden;
    }
    const int L = M->n_layers;
    return gemm(TC_F32_BIAS, B, M->K, xd, x, xd, M->wb[L], xd, M->logits, M->K, M->b[L], nullptr, s);
}

slos_status_t surr_forward(surr_model_t M, const float *phases, int B, float *probs, void *stream) {
    if (!M || !phases || !probs) return fail(SLOS_ERR_INVALID_ARG, "surr_forward: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    slos_status_t st = forward_impl(M, phases, B, s);
    if (st) return st;
    ProfScope ps("surr_softmax", 8.0 * B * M->K, s);
    softmax_kl_kernel<<<B, 256, 0, s>>>(M->logits, nullptr, M->K, 0.f, nullptr, nullptr, probs);
    return launch_check("softmax");
}

slos_status_t surr_train_step(surr_model_t M, const float *phases, const float *target, int B, float lr,
                              float *loss_rows, void *stream) {
    if (!M || !phases || !target) return fail(SLOS_ERR_INVALID_ARG, "surr_train_step: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    slos_status_t st = forward_impl(M, phases, B, s);
    if (st) return st;
    {
        ProfScope ps("surr_softmax", 12.0 * B * M->K, s);
        softmax_kl_kernel<<<B, 256, 0, s>>>(M->logits, target, M->K, 1.0f / B, M->dlog, loss_rows ? loss_rows : M->loss_rows,
                                            nullptr);
    }
    if ((st = launch_check("softmax_kl"))) return st;
    // backward through the layers: g = dL/d(pre-activation of layer l), [B][fan_out]
    const int L = M->n_layers;
    const __nv_bfloat16 *g = M->dlog;
    for (int l = L; l >= 0; --l) {
        const int fi = M->fan_in[l], fo = M->fan_out[l];
        const __nv_bfloat16 *xin = l == 0 ? M->x0 : M->h[l - 1];
        // weight gradient dW[fo][fi] = g^T x : A = g^T [fo][B], B = x^T [fi][B]
        if ((st = transpose(g, B, fo, M->tA, s))) return st;
        if ((st = transpose(xin, B, fi, M->tB, s))) return st;
        if ((st = gemm(TC_F32, fo, fi, B, M->tA, B, M->tB, B, M->gw[l], fi, nullptr, nullptr, s))) return st;
        {
            ProfScope ps("surr_colsum", 2.0 * B * fo, s);
            colsum_kernel<<<(fo + 255) / 256, 256, 0, s>>>(g, B, fo, M->gb[l]);
        }
        if ((st = launch_check("colsum"))) return st;
        if (l > 0) {
            // input gradient through GELU: dz_{l-1} = (g W_l) * gelu'(z_{l-1}); B operand = W_l^T [fi][fo]
            __nv_bfloat16 *dst = M->dh[l & 1];
            if ((st = gemm(TC_GELU_BWD, B, fi, fo, g, fo, M->wbt[l], fo, dst, fi, nullptr, M->z[l - 1], s))) return st;
            g = dst;
        }
    }
    // Adam
    M->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f / (1.f - std::pow(b1, (float)M->step)), c2 = 1.f / (1.f - std::pow(b2, (float)M->step));
    for (int l = 0; l <= L; ++l) {
        const int fi = M->fan_in[l], fo = M->fan_out[l];
        AdamArgs a{M->w[l], M->mw[l], M->vw[l], M->gw[l], M->wb[l], M->wbt[l], (int64_t)fi * fo, fo, fi, lr, b1, b2, 1e-8f, c1, c2};
        {
            ProfScope ps("surr_adam", 22.0 * fi * fo, s);
            adam_kernel<<<(unsigned)((a.n + 255) / 256), 256, 0, s>>>(a);
        }
        AdamArgs ab{M->b[l], M->mb[l], M->vb[l], M->gb[l], nullptr, nullptr, (int64_t)fo, 1, fo, lr, b1, b2, 1e-8f, c1, c2};
        adam_kernel<<<(fo + 255) / 256, 256, 0, s>>>(ab);
        count_launch();
        if ((st = launch_check("adam"))) return st;
    }
    return SLOS_OK;
}

slos_status_t surr_get_param(surr_model_t M, int layer, float *w_host, float *b_host) {
    if (!M || layer < 0 || layer > M->n_layers) return fail(SLOS_ERR_INVALID_ARG, "surr_get_param: layer");
    const size_t nw = (size_t)M->fan_in[layer] * M->fan_out[layer];
    if (w_host && cudaMemcpy(w_host, M->w[layer], nw * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(SLOS_ERR_CUDA, "surr_get_param: copy");
    if (b_host && cudaMemcpy(b_host, M->b[layer], M->fan_out[layer] * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(SLOS_ERR_CUDA, "surr_get_param: copy");
    return SLOS_OK;
}

slos_status_t surr_get_grad(surr_model_t M, int layer, float *gw_host, float *gb_host) {
    if (!M || layer < 0 || layer > M->n_layers) return fail(SLOS_ERR_INVALID_ARG, "surr_get_grad: layer");
    const size_t nw = (size_t)M->fan_in[layer] * M->fan_out[layer];
    if (gw_host && cudaMemcpy(gw_host, M->gw[layer], nw * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(SLOS_ERR_CUDA, "surr_get_grad: copy");
    if (gb_host && cudaMemcpy(gb_host, M->gb[layer], M->fan_out[layer] * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(SLOS_ERR_CUDA, "surr_get_grad: copy");
    return SLOS_OK;
}

slos_status_t surr_set_param(surr_model_t M, int layer, const float *w_host, const float *b_host) {
    if (!M || layer < 0 || layer > M->n_layers) return fail(SLOS_ERR_INVALID_ARG, "surr_set_param: layer");
    const int fi = M->fan_in[layer], fo = M->fan_out[layer];
    const size_t nw = (size_t)fi * fo;
    if (w_host) {
        cudaMemcpy(M->w[layer], w_host, nw * 4, cudaMemcpyHostToDevice);
        std::vector<__nv_bfloat16> hb(nw), hbt(nw);
        for (size_t i = 0; i < nw; ++i) {
            hb[i] = __float2bfloat16(w_host[i]);
            hbt[(i % fi) * fo + i / fi] = hb[i];
        }
        cudaMemcpy(M->wb[layer], hb.data(), nw * 2, cudaMemcpyHostToDevice);
        cudaMemcpy(M->wbt[layer], hbt.data(), nw * 2, cudaMemcpyHostToDevice);
    }
    if (b_host) cudaMemcpy(M->b[layer], b_host, fo * 4, cudaMemcpyHostToDevice);
    return SLOS_OK;
}

// Training checkpoint: a little-endian binary file
//   "SURRCKP1", int32 n_phases, hidden, n_layers, K, int32 step, float lr,
//   int64 stream_index, then per layer l = 0..n_layers: W, b, m_W, v_W, m_b, v_b (float32)
// (FP32 master weights and Adam moments; the BF16 copies are rebuilt on load).
slos_status_t surr_save(surr_model_t M, const char *path, int64_t stream_index) {
    if (!M || !path) return fail(SLOS_ERR_INVALID_ARG, "surr_save: NULL argument");
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(SLOS_ERR_CUDA, "surr_save: device error");
    FILE *f = fopen(path, "wb");
    if (!f) return fail(SLOS_ERR_INVALID_ARG, std::string("surr_save: cannot open ") + path);
    bool ok = fwrite("SURRCKP1", 1, 8, f) == 8;
    const int32_t hdr[5] = {M->n_phases, M->hidden, M->n_layers, M->K, M->step};
    ok = ok && fwrite(hdr, 4, 5, f) == 5 && fwrite(&M->lr, 4, 1, f) == 1 && fwrite(&stream_index, 8, 1, f) == 1;
    std::vector<float> h;
    for (int l = 0; ok && l <= M->n_layers; ++l) {
        const size_t nw = (size_t)M->fan_in[l] * M->fan_out[l], nb = (size_t)M->fan_out[l];
        const float *arrs[6] = {M->w[l], M->b[l], M->mw[l], M->vw[l], M->mb[l], M->vb[l]};
        const size_t lens[6] = {nw, nb, nw, nw, nb, nb};
        for (int q = 0; ok && q < 6; ++q) {
            h.resize(lens[q]);
            ok = cudaMemcpy(h.data(), arrs[q], lens[q] * 4, cudaMemcpyDeviceToHost) == cudaSuccess &&
                 fwrite(h.data(), 4, lens[q], f) == lens[q];
        }
    }
    ok = (fclose(f) == 0) && ok;
    return ok ? SLOS_OK : fail(SLOS_ERR_INTERNAL, std::string("surr_save: writing ") + path + " failed");
}

slos_status_t surr_load(surr_model_t M, const char *path, int64_t *stream_index) {
    if (!M || !path) return fail(SLOS_ERR_INVALID_ARG, "surr_load: NULL argument");
    FILE *f = fopen(path, "rb");
    if (!f) return fail(SLOS_ERR_INVALID_ARG, std::string("surr_load: cannot open ") + path);
    char magic[8];
    int32_t hdr[5];
    float lr = 0.f;
    int64_t idx = 0;
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "SURRCKP1", 8) == 0 && fread(hdr, 4, 5, f) == 5 &&
              fread(&lr, 4, 1, f) == 1 && fread(&idx, 8, 1, f) == 1;
    if (!ok) {
        fclose(f);
        return fail(SLOS_ERR_INVALID_ARG, std::string("surr_load: ") + path + " is not a surrogate checkpoint");
    }
    if (hdr[0] != M->n_phases || hdr[1] != M->hidden || hdr[2] != M->n_layers || hdr[3] != M->K) {
        fclose(f);
        return fail(SLOS_ERR_INVALID_ARG, "surr_load: the checkpoint's model dimensions differ from this model's");
    }
    std::vector<float> h;
    for (int l = 0; ok && l <= M->n_layers; ++l) {
        const size_t nw = (size_t)M->fan_in[l] * M->fan_out[l], nb = (size_t)M->fan_out[l];
        float *arrs[6] = {M->w[l], M->b[l], M->mw[l], M->vw[l], M->mb[l], M->vb[l]};
        const size_t lens[6] = {nw, nb, nw, nw, nb, nb};
        for (int q = 0; ok && q < 6; ++q) {
            h.resize(lens[q]);
            ok = fread(h.data(), 4, lens[q], f) == lens[q] &&
                 cudaMemcpy(arrs[q], h.data(), lens[q] * 4, cudaMemcpyHostToDevice) == cudaSuccess;
            if (ok && q == 0) {
                // BF16 copies of W and W^T, as the Adam kernel writes them
                const int fi = M->fan_in[l], fo = M->fan_out[l];
                std::vector<__nv_bfloat16> hb(nw), hbt(nw);
                for (size_t i = 0; i < nw; ++i) {
                    hb[i] = __float2bfloat16(h[i]);
                    hbt[(i % fi) * fo + i / fi] = hb[i];
                }
                ok = cudaMemcpy(M->wb[l], hb.data(), nw * 2, cudaMemcpyHostToDevice) == cudaSuccess &&
                     cudaMemcpy(M->wbt[l], hbt.data(), nw * 2, cudaMemcpyHostToDevice) == cudaSuccess;
            }
        }
    }
    fclose(f);
    if (!ok) return fail(SLOS_ERR_INVALID_ARG, std::string("surr_load: ") + path + " is truncated");
    M->step = hdr[4];
    M->lr = lr;
    if (stream_index) *stream_index = idx;
    return SLOS_OK;
}

slos_status_t surr_tv_rows(const float *q, const int *rows, const float *p, int n, int K, float *tv, void *stream) {
    if (n <= 0) return SLOS_OK;
    if (!q || !rows || !p || !tv) return fail(SLOS_ERR_INVALID_ARG, "surr_tv_rows: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    ProfScope ps("surr_tv", 8.0 * n * K, s);
    tv_rows_kernel<<<n, 256, 0, s>>>(q, rows, p, K, tv);
    return launch_check("tv_rows");
}

slos_status_t surr_screen(const float *q, int B, int K, const uint8_t *occ, int m, const void *U, const int *input_state,
                          float tol, float *marg_scratch, int *flag, void *stream) {
    if (B <= 0) return SLOS_OK;
    if (m < 1 || m > 24 || !q || !occ || !U || !input_state || !marg_scratch || !flag)
        return fail(SLOS_ERR_INVALID_ARG, "surr_screen: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    {
        ProfScope ps("surr_marginals", 4.0 * B * K + (double)K * m, s);
        marginals_kernel<<<B, 256, 0, s>>>(q, K, occ, m, marg_scratch);
    }
    slos_status_t st = launch_check("marginals");
    if (st) return st;
    ScreenArgs a;
    a.U = reinterpret_cast<const float2 *>(U);
    a.marg = marg_scratch;
    a.B = B;
    a.m = m;
    for (int i = 0; i < 24; ++i) a.s[i] = i < m ? (float)input_state[i] : 0.f;
    a.tol = tol;
    a.flag = flag;
    ProfScope ps("surr_screen", 8.0 * B * m * m, s);
    screen_kernel<<<(B + 127) / 128, 128, 0, s>>>(a);
    return launch_check("screen");
}

slos_status_t surr_scatter_rows(const float *src, const int *rows, int n, int K, float *dst, void *stream) {
    if (n <= 0) return SLOS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    ProfScope ps("surr_scatter", 8.0 * n * K, s);
    scatter_rows_kernel<<<n, 256, 0, s>>>(src, rows, K, dst);
    return launch_check("scatter_rows");
}

slos_status_t surr_gather_rows(const float *src, const int *rows, int n, int W, float *dst, void *stream) {
    if (n <= 0) return SLOS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    ProfScope ps("surr_gather", 8.0 * n * W, s);
    gather_rows_kernel<<<n, 128, 0, s>>>(src, rows, W, dst);
    return launch_check("gather_rows");
}

}  // extern "C"
