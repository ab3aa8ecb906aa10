// SLOS photon-number layer kernels (forward, backward, seed preparation).
//
// Data layout.  The batch is split into groups of 32 instances; lane l of a
// warp owns instance 32*g + l.  Photon-number layer k of group g is stored as
// complex64 [F_k][32] (state-major, instance-minor), so for a given Fock state
// all 32 lanes touch one contiguous 256-byte row: every gather of a parent or
// child amplitude is a fully coalesced load whose index is uniform across the
// warp, and the index arithmetic is done once per warp for 32 instances (the
// transition structure is shared by the batch, only the U coefficients differ,
// as in Sec. II-A.3).  Each warp walks a chunk of consecutive states, stepping
// the bar representation with next_bars() instead of re-ranking.
#pragma once

#include "common.cuh"

namespace slos {

enum Epilogue : int {
    EPI_STORE = 0,   // intermediate layer: write a_k
    EPI_PROBS = 1,   // final layer: p(t) = |a_n|^2 prod t! / prod s!  -> out [B][K]
    EPI_AMPS = 2,    // final layer: a_n * sqrt(prod t! / prod s!)     -> out [B][K] c64
    EPI_THRESH = 3,  // final layer: q(pattern(t)) += p(t)                -> out [B][Kq]
};

enum Seed : int {
    SEED_G = 0,            // k < n: read G_k
    SEED_PROBS_BCAST = 1,  // k == n: dL/dp shared by the batch, float [K]
    SEED_PROBS_T = 2,      // k == n: dL/dp per instance, transposed float [NG][F_n][32]
    SEED_AMPS_T = 3,       // k == n: dL/d(amp) per instance, transposed c64 [NG][F_n][32]
};

struct FwdArgs {
    const float2 *prev;  // a_{k-1}: [NG][Fprev][32]; unused when k == 1
    float2 *next;        // a_k: [NG][Fk][32]; may be null for the final layer
    const float2 *U;     // [B][m][m]
    void *out;           // final-layer output [B][K]
    int64_t Fk, Fprev, K;
    int m, k, col, B, NG, chunk;
    float inv_sfact;
    int pat_off[kMaxPhotons + 2];  // threshold: first index of patterns with |b| = i
};

struct BwdArgs {
    const float2 *aprev;  // a_{k-1}: [NG][Fprev][32]; unused when k == 1
    const float2 *Gk;     // G_k: [NG][Fk][32] (k < n)
    float2 *Gprev;        // G_{k-1}: [NG][Fprev][32] (k > 1)
    const float2 *an;     // a_n: [NG][Fk][32] (k == n)
    const void *seed;     // see Seed
    const float2 *U;      // [B][m][m]
    float2 *dUpart;       // [NG][gridDim.x][32][m]
    int64_t Fk, Fprev;
    int m, k, col, B, NG, chunk;
    float inv_sfact;
};

struct PrepArgs {
    const void *dout;    // [B][stride] float or c64
    int64_t stride;      // elements between instances (0 = shared)
    void *outT;          // [NG][Fn][32] float or c64
    int64_t Fn;
    int m, n, B, NG, chunk, kind;  // kind: 0 PNR probs, 1 amps, 2 threshold
    int pat_off[kMaxPhotons + 2];
};

constexpr int kWarpsPerBlock = 8;
constexpr int kThreads = kWarpsPerBlock * 32;

// ------------------------------------------------------------------ forward
template <int MMAX, int EPI, bool SAVE>
__global__ void __launch_bounds__(kThreads) slos_fwd_kernel(FwdArgs a) {
    extern __shared__ float4 smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int grp = blockIdx.y;
    const int inst = grp * kLanes + lane;
    const bool valid = inst < a.B;
    const int m = a.m;
    const int L = a.k + m - 1;

    float2 u[MMAX];
#pragma unroll
    for (int j = 0; j < MMAX; ++j) {
        u[j] = make_float2(0.f, 0.f);
        if (j < m && valid) u[j] = a.U[((int64_t)inst * m + j) * m + a.col];
    }

    const int64_t gprev = (int64_t)grp * a.Fprev;
    const int64_t gnext = (int64_t)grp * a.Fk;
    const int64_t nchunks = (a.Fk + a.chunk - 1) / a.chunk;
    const int64_t wstride = (int64_t)gridDim.x * kWarpsPerBlock;

    // per-warp staging tile for the [B][K] output: tile[lane(instance)][33]
    float *tile = reinterpret_cast<float *>(smem_raw) + warp * (32 * 33 * (EPI == EPI_AMPS ? 2 : 1));

    for (int64_t ch = (int64_t)blockIdx.x * kWarpsPerBlock + warp; ch < nchunks; ch += wstride) {
        const int64_t c0 = ch * a.chunk;
        const int64_t c1 = min(c0 + (int64_t)a.chunk, a.Fk);
        int p[MMAX];
        unrank_bars<MMAX>(c0, m, L, p);
        int run_pat = -1;
        float run_val = 0.f;
        for (int64_t c = c0; c < c1; ++c) {
            float2 acc = make_float2(0.f, 0.f);
            int64_t S = 0;
            float fprod = 1.f;
            uint32_t supp = 0;
#pragma unroll
            for (int j = 0; j < MMAX; ++j) {
                if (j < m) {
                    const int tj = occupation<MMAX>(j, m, L, p);
                    if (tj > 0) {
                        float2 v;
                        if (a.k == 1) {
                            v = make_float2(1.f, 0.f);
                        } else {
                            v = __ldg(&a.prev[(gprev + (c - S)) * kLanes + lane]);
                        }
                        acc = cfma(u[j], v, acc);
                        if (EPI != EPI_STORE) {
                            fprod *= c_fact.v[tj];
                            supp |= 1u << j;
                        }
                    }
                    if (j < m - 1) S += (int64_t)binom_m1(p[j], m - 2 - j);
                }
            }
            if (SAVE || EPI == EPI_STORE) a.next[(gnext + c) * kLanes + lane] = acc;
            if (EPI == EPI_PROBS) {
                const float w = fprod * a.inv_sfact;
                tile[lane * 33 + (int)(c - c0)] = w * (acc.x * acc.x + acc.y * acc.y);
            } else if (EPI == EPI_AMPS) {
                const float sw = sqrtf(fprod * a.inv_sfact);
                float2 *t2 = reinterpret_cast<float2 *>(tile);
                t2[lane * 33 + (int)(c - c0)] = cscale(acc, sw);
            } else if (EPI == EPI_THRESH) {
                const float w = fprod * a.inv_sfact;
                const float pr = w * (acc.x * acc.x + acc.y * acc.y);
                const int pat = a.pat_off[__popc(supp)] + (int)colex_rank(supp);
                if (pat != run_pat) {
                    if (run_pat >= 0 && valid)
                        atomicAdd(reinterpret_cast<float *>(a.out) + (int64_t)inst * a.K + run_pat, run_val);
                    run_pat = pat;
                    run_val = 0.f;
                }
                run_val += pr;
            }
            next_bars<MMAX>(m, L, p);
        }
        if (EPI == EPI_THRESH) {
            if (run_pat >= 0 && valid)
                atomicAdd(reinterpret_cast<float *>(a.out) + (int64_t)inst * a.K + run_pat, run_val);
        }
        if (EPI == EPI_PROBS || EPI == EPI_AMPS) {
            __syncwarp();
            const int nc = (int)(c1 - c0);
            for (int i = 0; i < kLanes; ++i) {
                const int ii = grp * kLanes + i;
                if (ii < a.B && lane < nc) {
                    if (EPI == EPI_PROBS) {
                        reinterpret_cast<float *>(a.out)[(int64_t)ii * a.K + c0 + lane] = tile[i * 33 + lane];
                    } else {
                        const float2 *t2 = reinterpret_cast<const float2 *>(tile);
                        reinterpret_cast<float2 *>(a.out)[(int64_t)ii * a.K + c0 + lane] = t2[i * 33 + lane];
                    }
                }
            }
            __syncwarp();
        }
    }
}

// ------------------------------------------------------------------ backward
// Layer k: for every parent t' in F_{k-1} and every mode j (all children
// t' + e_j exist):
//      G_{k-1}(t') = sum_j conj(U[j, c_k]) G_k(t' + e_j)
//      dU[j, c_k] += conj(a_{k-1}(t')) G_k(t' + e_j)
// For k == n the child gradient is formed on the fly from a_n and the output
// gradient (seed).
template <int MMAX, int SEED>
__global__ void __launch_bounds__(kThreads) slos_bwd_kernel(BwdArgs a) {
    __shared__ float2 red[kWarpsPerBlock][32];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int grp = blockIdx.y;
    const int inst = grp * kLanes + lane;
    const bool valid = inst < a.B;
    const int m = a.m;
    const int L = (a.k - 1) + m - 1;  // parent layer string length

    float2 u[MMAX], dU[MMAX];
#pragma unroll
    for (int j = 0; j < MMAX; ++j) {
        u[j] = make_float2(0.f, 0.f);
        dU[j] = make_float2(0.f, 0.f);
        if (j < m && valid) u[j] = a.U[((int64_t)inst * m + j) * m + a.col];
    }
    const int64_t gprev = (int64_t)grp * a.Fprev;
    const int64_t gk = (int64_t)grp * a.Fk;
    const int64_t nchunks = (a.Fprev + a.chunk - 1) / a.chunk;
    const int64_t wstride = (int64_t)gridDim.x * kWarpsPerBlock;

    for (int64_t ch = (int64_t)blockIdx.x * kWarpsPerBlock + warp; ch < nchunks; ch += wstride) {
        const int64_t c0 = ch * a.chunk;
        const int64_t c1 = min(c0 + (int64_t)a.chunk, a.Fprev);
        int p[MMAX];
        unrank_bars<MMAX>(c0, m, L, p);
        for (int64_t c = c0; c < c1; ++c) {
            const float2 av = (a.k == 1) ? make_float2(1.f, 0.f) : __ldg(&a.aprev[(gprev + c) * kLanes + lane]);
            float fp = 1.f;
            if (SEED != SEED_G) {
#pragma unroll
                for (int j = 0; j < MMAX; ++j)
                    if (j < m) fp *= c_fact.v[occupation<MMAX>(j, m, L, p)];
            }
            float2 gacc = make_float2(0.f, 0.f);
            int64_t S = 0;
#pragma unroll
            for (int j = 0; j < MMAX; ++j) {
                if (j < m) {
                    const int64_t cidx = c + S;
                    const int64_t off = (gk + cidx) * kLanes + lane;
                    float2 g;
                    if (SEED == SEED_G) {
                        g = __ldg(&a.Gk[off]);
                    } else {
                        const int tj = occupation<MMAX>(j, m, L, p);
                        const float w = fp * (float)(tj + 1) * a.inv_sfact;
                        const float2 an = __ldg(&a.an[off]);
                        if (SEED == SEED_PROBS_BCAST) {
                            const float dp = __ldg(reinterpret_cast<const float *>(a.seed) + cidx);
                            g = cscale(an, 2.f * dp * w);
                        } else if (SEED == SEED_PROBS_T) {
                            const float dp = __ldg(reinterpret_cast<const float *>(a.seed) + off);
                            g = cscale(an, 2.f * dp * w);
                        } else {
                            const float2 d = __ldg(reinterpret_cast<const float2 *>(a.seed) + off);
                            g = cscale(d, sqrtf(w));
                        }
                    }
                    gacc = cfma_conj_a(u[j], g, gacc);
                    dU[j] = cfma_conj_a(av, g, dU[j]);
                    if (j < m - 1) S += (int64_t)binom(p[j], m - 2 - j);
                }
            }
            if (a.k > 1) a.Gprev[(gprev + c) * kLanes + lane] = gacc;
            next_bars<MMAX>(m, L, p);
        }
    }
    // reduce dU over the warps of this block, one mode at a time
    float2 *dst = a.dUpart + (((int64_t)grp * gridDim.x + blockIdx.x) * kLanes) * m;
#pragma unroll
    for (int j = 0; j < MMAX; ++j) {
        if (j < m) {
            red[warp][lane] = dU[j];
            __syncthreads();
            if (warp == 0) {
                float2 s = red[0][lane];
#pragma unroll
                for (int w = 1; w < kWarpsPerBlock; ++w) {
                    s.x += red[w][lane].x;
                    s.y += red[w][lane].y;
                }
                dst[lane * m + j] = s;
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------------ seed prep
// Gathers the output gradient into the state-major layout of layer n:
// outT[g][t][lane] = dout[inst][idx(t)], idx(t) = t (PNR, amps) or the
// threshold pattern of t.
template <int MMAX>
__global__ void __launch_bounds__(kThreads) slos_seed_prep_kernel(PrepArgs a) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int grp = blockIdx.y;
    const int inst = grp * kLanes + lane;
    const bool valid = inst < a.B;
    const int m = a.m;
    const int L = a.n + m - 1;
    const int64_t nchunks = (a.Fn + a.chunk - 1) / a.chunk;
    const int64_t wstride = (int64_t)gridDim.x * kWarpsPerBlock;
    const int64_t base = (int64_t)grp * a.Fn;
    for (int64_t ch = (int64_t)blockIdx.x * kWarpsPerBlock + warp; ch < nchunks; ch += wstride) {
        const int64_t c0 = ch * a.chunk;
        const int64_t c1 = min(c0 + (int64_t)a.chunk, a.Fn);
        int p[MMAX];
        unrank_bars<MMAX>(c0, m, L, p);
        for (int64_t c = c0; c < c1; ++c) {
            int64_t idx = c;
            if (a.kind == 2) {
                uint32_t supp = 0;
#pragma unroll
                for (int j = 0; j < MMAX; ++j)
                    if (j < m && occupation<MMAX>(j, m, L, p) > 0) supp |= 1u << j;
                idx = a.pat_off[__popc(supp)] + (int64_t)colex_rank(supp);
            }
            const int64_t src = (valid ? (int64_t)inst * a.stride : 0) + idx;
            if (a.kind == 1) {
                float2 v = valid ? __ldg(reinterpret_cast<const float2 *>(a.dout) + src) : make_float2(0.f, 0.f);
                reinterpret_cast<float2 *>(a.outT)[(base + c) * kLanes + lane] = v;
            } else {
                float v = valid ? __ldg(reinterpret_cast<const float *>(a.dout) + src) : 0.f;
                reinterpret_cast<float *>(a.outT)[(base + c) * kLanes + lane] = v;
            }
            next_bars<MMAX>(m, L, p);
        }
    }
}

// ------------------------------------------------------------------ launchers
inline size_t fwd_smem_bytes(int epi) {
    if (epi == EPI_PROBS) return (size_t)kWarpsPerBlock * 32 * 33 * sizeof(float);
    if (epi == EPI_AMPS) return (size_t)kWarpsPerBlock * 32 * 33 * sizeof(float2);
    return 0;
}

// Defines the host launchers of one MMAX instantiation (one per .cu file so
// the instantiations compile in parallel).
#define SLOS_DEFINE_LAUNCHERS(MM)                                                                            \
    cudaError_t slos_init_m##MM() {                                                                          \
        const int sm = (int)fwd_smem_bytes(EPI_AMPS);                                                        \
        cudaError_t e = cudaFuncSetAttribute(slos_fwd_kernel<MM, EPI_AMPS, false>,                          \
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, sm);               \
        if (e != cudaSuccess) return e;                                                                      \
        return cudaFuncSetAttribute(slos_fwd_kernel<MM, EPI_AMPS, true>,                                    \
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, sm);                        \
    }                                                                                                        \
    cudaError_t slos_launch_fwd_m##MM(const FwdArgs &a, int epi, bool save, int blocks_x, cudaStream_t s) { \
        dim3 grid(blocks_x, a.NG);                                                                           \
        const size_t sm = fwd_smem_bytes(epi);                                                               \
        switch (epi * 2 + (save ? 1 : 0)) {                                                                  \
            case 0:                                                                                          \
            case 1: slos_fwd_kernel<MM, EPI_STORE, true><<<grid, kThreads, 0, s>>>(a); break;               \
            case 2: slos_fwd_kernel<MM, EPI_PROBS, false><<<grid, kThreads, sm, s>>>(a); break;             \
            case 3: slos_fwd_kernel<MM, EPI_PROBS, true><<<grid, kThreads, sm, s>>>(a); break;              \
            case 4: slos_fwd_kernel<MM, EPI_AMPS, false><<<grid, kThreads, sm, s>>>(a); break;              \
            case 5: slos_fwd_kernel<MM, EPI_AMPS, true><<<grid, kThreads, sm, s>>>(a); break;               \
            case 6: slos_fwd_kernel<MM, EPI_THRESH, false><<<grid, kThreads, 0, s>>>(a); break;             \
            case 7: slos_fwd_kernel<MM, EPI_THRESH, true><<<grid, kThreads, 0, s>>>(a); break;              \
            default: return cudaErrorInvalidValue;                                                           \
        }                                                                                                    \
        return cudaGetLastError();                                                                           \
    }                                                                                                        \
    cudaError_t slos_launch_bwd_m##MM(const BwdArgs &a, int seed, int blocks_x, cudaStream_t s) {           \
        dim3 grid(blocks_x, a.NG);                                                                           \
        switch (seed) {                                                                                      \
            case SEED_G: slos_bwd_kernel<MM, SEED_G><<<grid, kThreads, 0, s>>>(a); break;                   \
            case SEED_PROBS_BCAST: slos_bwd_kernel<MM, SEED_PROBS_BCAST><<<grid, kThreads, 0, s>>>(a); break; \
            case SEED_PROBS_T: slos_bwd_kernel<MM, SEED_PROBS_T><<<grid, kThreads, 0, s>>>(a); break;       \
            case SEED_AMPS_T: slos_bwd_kernel<MM, SEED_AMPS_T><<<grid, kThreads, 0, s>>>(a); break;         \
            default: return cudaErrorInvalidValue;                                                           \
        }                                                                                                    \
        return cudaGetLastError();                                                                           \
    }                                                                                                        \
    cudaError_t slos_launch_prep_m##MM(const PrepArgs &a, int blocks_x, cudaStream_t s) {                   \
        dim3 grid(blocks_x, a.NG);                                                                           \
        slos_seed_prep_kernel<MM><<<grid, kThreads, 0, s>>>(a);                                              \
        return cudaGetLastError();                                                                           \
    }

#define SLOS_DECLARE_LAUNCHERS(MM)                                                                  \
    cudaError_t slos_init_m##MM();                                                                  \
    cudaError_t slos_launch_fwd_m##MM(const FwdArgs &a, int epi, bool save, int blocks_x, cudaStream_t s); \
    cudaError_t slos_launch_bwd_m##MM(const BwdArgs &a, int seed, int blocks_x, cudaStream_t s);  \
    cudaError_t slos_launch_prep_m##MM(const PrepArgs &a, int blocks_x, cudaStream_t s);

}  // namespace slos
