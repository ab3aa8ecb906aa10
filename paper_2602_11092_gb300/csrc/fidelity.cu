// Fidelity kernel (kernel-methods section): with the embedding
// |phi(x)> = U(x)|s> of a Fock input s,
//     K[i][j] = |<phi_a(i)|phi_b(j)>|^2 = |<s|Ua[i]^dag Ub[j]|s>|^2,
// and for a Fock state <s|V|s> = Per(W) / prod_i s_i! with the n x n matrix
// W[a][b] = V[c_a][c_b] = sum_k conj(Ua[i][k][c_a]) Ub[j][k][c_b] over the
// photon columns c_1 <= ... <= c_n.
//
// One thread per pair (i, j) in 16 x 16 tiles; the photon columns of the
// tile's 16 + 16 unitaries are staged in shared memory.  W is formed in FP32
// (each entry an m-term inner product) and kept in registers; the permanent
// uses Glynn's formula
//     Per(W) = 2^(1-n) sum_{delta in {+-1}^n, delta_1 = 1} (prod_a delta_a)
//              prod_b (sum_a delta_a W[a][b])
// walked in Gray-code order (one row sum update per term) with the row sums,
// products and the signed total in double-float arithmetic (dfloat.cuh, about
// 44 bits on the FP32 pipe): the terms reach about n^n / 2^(n-1) while the
// permanent of a block of a unitary is at most 1, so FP32 sums would lose the
// result.  The updates add +-2 W[r][c], exact in float.  n <= 8 keeps W in
// registers.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/slos.h"
#include "common.cuh"
#include "dfloat.cuh"
#include "profile.h"

namespace slos {
slos_status_t fail(slos_status_t st, const std::string &msg);

constexpr int kFidTile = 16;
constexpr int kFidMaxPhotons = 8;

struct FidArgs {
    const float2 *Ua, *Ub;
    float *K;
    int m, Na, Nb;
    int cols[kFidMaxPhotons];
    float inv_sf2;   // 1 / (prod s_i!)^2
};

template <int N>
__global__ void __launch_bounds__(kFidTile *kFidTile) fidelity_kernel(FidArgs a) {
    extern __shared__ float2 sm[];
    const int m = a.m;
    float2 *wa = sm;                              // [16][m][N]
    float2 *wb = sm + (size_t)kFidTile * m * N;   // [16][m][N]
    const int i0 = blockIdx.y * kFidTile, j0 = blockIdx.x * kFidTile;
    const int tid = threadIdx.y * kFidTile + threadIdx.x;
    const int per = m * N;
    for (int idx = tid; idx < kFidTile * per; idx += kFidTile * kFidTile) {
        const int t = idx / per, r = idx % per, k = r / N, c = r % N;
        const int col = a.cols[c];
        wa[idx] = (i0 + t < a.Na) ? a.Ua[((size_t)(i0 + t) * m + k) * m + col] : make_float2(0.f, 0.f);
        wb[idx] = (j0 + t < a.Nb) ? a.Ub[((size_t)(j0 + t) * m + k) * m + col] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int i = i0 + threadIdx.y, j = j0 + threadIdx.x;
    if (i >= a.Na || j >= a.Nb) return;
    const float2 *pa = wa + (size_t)threadIdx.y * per, *pb = wb + (size_t)threadIdx.x * per;
    float2 W[N][N];
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = 0; c < N; ++c) W[r][c] = make_float2(0.f, 0.f);
    for (int k = 0; k < m; ++k) {
#pragma unroll
        for (int r = 0; r < N; ++r) {
            const float2 x = pa[k * N + r];
#pragma unroll
            for (int c = 0; c < N; ++c) W[r][c] = cfma_conj_a(x, pb[k * N + c], W[r][c]);
        }
    }
    // Glynn, Gray-code order over delta_2..delta_N (bit q-1 of d: delta_{q+1} = -1)
    cdfl S[N];
#pragma unroll
    for (int c = 0; c < N; ++c) {
        S[c] = {df_zero(), df_zero()};
#pragma unroll
        for (int r = 0; r < N; ++r) {
            S[c].re = df_add_f(S[c].re, W[r][c].x);
            S[c].im = df_add_f(S[c].im, W[r][c].y);
        }
    }
    auto product = [&]() {
        cdfl pr = S[0];
#pragma unroll
        for (int c = 1; c < N; ++c) pr = cdf_mul(pr, S[c]);
        return pr;
    };
    cdfl t = product();
    uint32_t d = 0;
    for (uint32_t g = 1; g < (1u << (N - 1)); ++g) {
        const int q = __ffs(g);  // flips delta_{q+1}, row q of W (1-based bit index q)
        d ^= 1u << (q - 1);
        const float sgn = ((d >> (q - 1)) & 1u) ? -2.f : 2.f;
#pragma unroll
        for (int r = 1; r < N; ++r) {
            if (r == q) {
#pragma unroll
                for (int c = 0; c < N; ++c) {
                    S[c].re = df_add_f(S[c].re, sgn * W[r][c].x);
                    S[c].im = df_add_f(S[c].im, sgn * W[r][c].y);
                }
            }
        }
        const cdfl pr = product();
        t = (__popc(d) & 1) ? cdf_sub(t, pr) : cdf_add(t, pr);
    }
    const float scale = 1.f / (float)(1u << (N - 1));
    const float tr = df_float(t.re) * scale, ti = df_float(t.im) * scale;
    a.K[(size_t)i * a.Nb + j] = (tr * tr + ti * ti) * a.inv_sf2;
}

template <int N>
static cudaError_t launch_fid(const FidArgs &a, cudaStream_t s) {
    dim3 grid((a.Nb + kFidTile - 1) / kFidTile, (a.Na + kFidTile - 1) / kFidTile);
    const size_t sm = 2 * (size_t)kFidTile * a.m * N * sizeof(float2);
    fidelity_kernel<N><<<grid, dim3(kFidTile, kFidTile), sm, s>>>(a);
    return cudaGetLastError();
}

}  // namespace slos

using namespace slos;

extern "C" {

slos_status_t slos_fidelity_kernel(int m, const int *input_state, const void *Ua, int Na, const void *Ub, int Nb,
                                   float *K, void *stream) {
    if (!input_state) return fail(SLOS_ERR_INVALID_ARG, "slos_fidelity_kernel: NULL input_state");
    if (m < 1 || m > kMaxModes) return fail(SLOS_ERR_UNSUPPORTED, "slos_fidelity_kernel: m must be in [1, 24]");
    if (Na < 0 || Nb < 0) return fail(SLOS_ERR_INVALID_ARG, "slos_fidelity_kernel: negative count");
    FidArgs a;
    int n = 0;
    double sf = 1.0;
    for (int i = 0; i < m; ++i) {
        if (input_state[i] < 0) return fail(SLOS_ERR_INVALID_ARG, "slos_fidelity_kernel: negative occupation");
        for (int q = 0; q < input_state[i]; ++q) {
            if (n >= kFidMaxPhotons)
                return fail(SLOS_ERR_UNSUPPORTED, "slos_fidelity_kernel: at most 8 photons");
            a.cols[n++] = i;
            sf *= (double)(q + 1);
        }
    }
    if (n == 0) return fail(SLOS_ERR_INVALID_ARG, "slos_fidelity_kernel: the input state holds no photon");
    if ((int64_t)(Na + kFidTile - 1) / kFidTile > 65535)
        return fail(SLOS_ERR_UNSUPPORTED, "slos_fidelity_kernel: at most 65535 * 16 rows");
    if (Na == 0 || Nb == 0) return SLOS_OK;
    if (!Ua || !Ub || !K) return fail(SLOS_ERR_INVALID_ARG, "slos_fidelity_kernel: NULL pointer");
    a.Ua = reinterpret_cast<const float2 *>(Ua);
    a.Ub = reinterpret_cast<const float2 *>(Ub);
    a.K = K;
    a.m = m;
    a.Na = Na;
    a.Nb = Nb;
    a.inv_sf2 = 1.0 / (sf * sf);
    cudaStream_t s = (cudaStream_t)stream;
    ProfScope ps("slos_fidelity", 8.0 * m * n * ((double)Na + Nb) + 4.0 * Na * Nb, s);
    cudaError_t e;
    switch (n) {
        case 1: e = launch_fid<1>(a, s); break;
        case 2: e = launch_fid<2>(a, s); break;
        case 3: e = launch_fid<3>(a, s); break;
        case 4: e = launch_fid<4>(a, s); break;
        case 5: e = launch_fid<5>(a, s); break;
        case 6: e = launch_fid<6>(a, s); break;
        case 7: e = launch_fid<7>(a, s); break;
        default: e = launch_fid<8>(a, s); break;
    }
    if (e != cudaSuccess) return fail(SLOS_ERR_CUDA, std::string("slos_fidelity_kernel: ") + cudaGetErrorString(e));
    return SLOS_OK;
}

}  // extern "C"
