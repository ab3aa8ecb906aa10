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
    EPI_THRESH = 3,  // final layer in list order: q(b) = sum of p(t) over the pattern's states -> out [B][Kq]
};
// (Threshold plans without tables store a_n with EPI_STORE; threshold.cu sums
// the patterns.)

// Output-gradient seed of the final backward layer.  The prep step folds the
// weight w_t = prod t_j! / prod s_i! into it, so that
//      probabilities / threshold: G_n(t) = seed(t) * a_n(t), seed = 2 w_t dL/dp(t)
//      amplitudes:                G_n(t) = seed(t),          seed = sqrt(w_t) dL/d(amp)
enum Seed : int {
    SEED_G = 0,       // k < n: read G_k
    SEED_BCAST = 1,   // k == n: float [F_n], the same for every instance
    SEED_T = 2,       // k == n: float [NG][F_n][32]
    SEED_AMPS_T = 3,  // k == n: complex64 [NG][F_n][32]
};

struct FwdArgs {
    const float2 *prev;  // a_{k-1}: [NG][Fprev][32]; unused when k == 1
    float2 *next;        // a_k: [NG][Fk][32]; may be null for the final layer
    const float2 *U;     // [B][m][m]
    void *out;           // final-layer output [B][K]
    int64_t Fk, Fprev, K;
    int m, k, col, B, NG, chunk;
    float inv_sfact;
    int *status;                   // plan status word (bounds checks of SLOS_DEBUG builds)
};

// Threshold outcomes from a stored a_n (threshold.cu).
struct ThreshArgs {
    const float2 *an;              // a_n: [NG][Fn][32]
    float *out;                    // [B][K]
    int64_t Fn, K;
    int m, n, B, NG, jmax;         // jmax = min(n, m): pattern classes |b| = 1..jmax
    float inv_sfact;
    int *status;                   // plan status word (bounds checks of SLOS_DEBUG builds)
};
cudaError_t slos_launch_thresh_sum(const ThreshArgs &a, cudaStream_t s);

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
    void *outT;          // [NG][Fn][32] float or c64, or [Fn] float (shared seed)
    int64_t Fn;
    int m, n, B, NG, chunk, kind;  // kind: 0 PNR probs, 1 amps, 2 threshold
    float inv_sfact;
    int pat_off[kMaxPhotons + 2];
};

constexpr int kWarpsPerBlock = 8;
constexpr int kCStore = 8;  // states per warp iteration, intermediate layers
constexpr int kCFinal = 8;  // final layer
constexpr int kCBwd = 4;    // parents per warp iteration, backward
constexpr int kThreads = kWarpsPerBlock * 32;

// ------------------------------------------------------------------ forward
// Each warp walks a chunk of consecutive Fock states of layer k, C states at a
// time.  The mode loop is outermost and warp-uniform (so U[j, c_k] of the
// lane's instance is a register), and for each mode the C states' parent
// loads are independent, which keeps 8+ coalesced 256-byte loads in flight
// per warp.  A state is carried as its bar mask; the next state is the next
// larger mask with the same popcount.
template <int MMAX, int EPI, bool SAVE, int C>
__global__ void __launch_bounds__(kThreads) slos_fwd_kernel(FwdArgs a) {
    using Z = typename BarMask<MMAX>::T;
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
    const float2 *prevg = a.prev + (int64_t)grp * a.Fprev * kLanes + lane;
    float2 *nextg = a.next + (int64_t)grp * a.Fk * kLanes + lane;
    const int64_t nchunks = (a.Fk + a.chunk - 1) / a.chunk;
    const int64_t wstride = (int64_t)gridDim.x * kWarpsPerBlock;
    float *tile = reinterpret_cast<float *>(smem_raw) + warp * (32 * 33 * (EPI == EPI_AMPS ? 2 : 1));

    for (int64_t ch = (int64_t)blockIdx.x * kWarpsPerBlock + warp; ch < nchunks; ch += wstride) {
        const int64_t c0 = ch * a.chunk;
        const int64_t c1 = min(c0 + (int64_t)a.chunk, a.Fk);
        Z z = unrank_mask<MMAX, Z>(c0, m, L);
        for (int64_t cb = c0; cb < c1; cb += C) {
            Z rem[C];
            int prevbar[C], S[C];
            float2 acc[C];
            float fp[C];
            bool live[C];
#pragma unroll
            for (int i = 0; i < C; ++i) {
                live[i] = cb + i < c1;
                rem[i] = z;
                z = next_comb(z);
                prevbar[i] = L;
                S[i] = 0;
                acc[i] = make_float2(0.f, 0.f);
                fp[i] = 1.f;
            }
#pragma unroll
            for (int i = 0; i < C; ++i)
                if (!live[i]) rem[i] = rem[0];  // keep index arithmetic in range
#pragma unroll
            for (int j = 0; j < MMAX; ++j) {
                if (j < m) {
#pragma unroll
                    for (int i = 0; i < C; ++i) {
                        int pb = -1;
                        if (j < m - 1) {
                            pb = top_bit(rem[i]);
                            rem[i] ^= (Z)1 << pb;
                        }
                        const int tj = prevbar[i] - pb - 1;
                        prevbar[i] = pb;
                        if (tj > 0 && live[i]) {
                            const float2 v = (a.k == 1) ? make_float2(1.f, 0.f)
                                                        : __ldg(prevg + (int64_t)(cb + i - S[i]) * kLanes);
                            acc[i] = cfma(u[j], v, acc[i]);
                            if (EPI != EPI_STORE) fp[i] *= c_fact.v[tj];
                        }
                        if (j < m - 1) S[i] += (int)binom_m1(pb, m - 2 - j);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < C; ++i) {
                if (!live[i]) continue;
                const int64_t c = cb + i;
                if (SAVE || EPI == EPI_STORE) nextg[c * kLanes] = acc[i];
                if (EPI == EPI_PROBS) {
                    tile[lane * 33 + (int)(c - c0)] = fp[i] * a.inv_sfact * (acc[i].x * acc[i].x + acc[i].y * acc[i].y);
                } else if (EPI == EPI_AMPS) {
                    float2 *t2 = reinterpret_cast<float2 *>(tile);
                    t2[lane * 33 + (int)(c - c0)] = cscale(acc[i], sqrtf(fp[i] * a.inv_sfact));
                }
            }
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

// Gradient of child state cidx (element offset `off` in the [NG][F_k][32]
// layout) for the reverse recursion.
template <int SEED>
__device__ __forceinline__ float2 load_child_grad(const BwdArgs &a, int64_t off, int64_t cidx) {
    if (SEED == SEED_G) return __ldg(a.Gk + off);
    if (SEED == SEED_AMPS_T) return __ldg(reinterpret_cast<const float2 *>(a.seed) + off);
    const float2 an = __ldg(a.an + off);
    const float sc = (SEED == SEED_BCAST) ? __ldg(reinterpret_cast<const float *>(a.seed) + cidx)
                                          : __ldg(reinterpret_cast<const float *>(a.seed) + off);
    return cscale(an, sc);
}

// ------------------------------------------------------------------ backward
// Layer k: for every parent t' in F_{k-1} and every mode j (all children
// t' + e_j exist):
//      G_{k-1}(t') = sum_j conj(U[j, c_k]) G_k(t' + e_j)
//      dU[j, c_k] += conj(a_{k-1}(t')) G_k(t' + e_j)
// For k == n the child gradient is formed on the fly from a_n and the output
// gradient (seed).  C parents per warp iteration, mode loop outermost.
template <int MMAX, int SEED, int C>
__global__ void __launch_bounds__(kThreads) slos_bwd_kernel(BwdArgs a) {
    using Z = typename BarMask<MMAX>::T;
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
    const int64_t gofs_prev = (int64_t)grp * a.Fprev * kLanes + lane;
    const int64_t gofs_k = (int64_t)grp * a.Fk * kLanes + lane;
    const int64_t nchunks = (a.Fprev + a.chunk - 1) / a.chunk;
    const int64_t wstride = (int64_t)gridDim.x * kWarpsPerBlock;

    for (int64_t ch = (int64_t)blockIdx.x * kWarpsPerBlock + warp; ch < nchunks; ch += wstride) {
        const int64_t c0 = ch * a.chunk;
        const int64_t c1 = min(c0 + (int64_t)a.chunk, a.Fprev);
        Z z = unrank_mask<MMAX, Z>(c0, m, L);
        for (int64_t cb = c0; cb < c1; cb += C) {
            Z rem[C];
            int prevbar[C], S[C];
            float2 av[C], gacc[C];
            bool live[C];
#pragma unroll
            for (int i = 0; i < C; ++i) {
                live[i] = cb + i < c1;
                rem[i] = z;
                z = next_comb(z);
                prevbar[i] = L;
                S[i] = 0;
                gacc[i] = make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int i = 0; i < C; ++i) {
                if (!live[i]) rem[i] = rem[0];
                av[i] = make_float2(0.f, 0.f);
                if (live[i]) av[i] = (a.k == 1) ? make_float2(1.f, 0.f) : __ldg(a.aprev + gofs_prev + (cb + i) * kLanes);
            }
#pragma unroll
            for (int j = 0; j < MMAX; ++j) {
                if (j < m) {
#pragma unroll
                    for (int i = 0; i < C; ++i) {
                        int pb = -1;
                        if (j < m - 1) {
                            pb = top_bit(rem[i]);
                            rem[i] ^= (Z)1 << pb;
                        }
                        const int tj = prevbar[i] - pb - 1;
                        prevbar[i] = pb;
                        const int64_t cidx = cb + i + S[i];
                        const int64_t off = gofs_k + cidx * kLanes;
                        (void)tj;
                        float2 g = make_float2(0.f, 0.f);
                        if (live[i]) g = load_child_grad<SEED>(a, off, cidx);
                        gacc[i] = cfma_conj_a(u[j], g, gacc[i]);
                        dU[j] = cfma_conj_a(av[i], g, dU[j]);
                        if (j < m - 1) S[i] += (int)binom(pb, m - 2 - j);
                    }
                }
            }
            if (a.k > 1) {
#pragma unroll
                for (int i = 0; i < C; ++i)
                    if (live[i]) a.Gprev[gofs_prev + (cb + i) * kLanes] = gacc[i];
            }
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
// Per-instance seeds in the state-major layout of layer n:
//   kind 0 (PNR probs):  outT[g][t][lane] = 2 w_t dout[inst][t]
//   kind 2 (threshold):  outT[g][t][lane] = 2 w_t dout[inst][pattern(t)]
//   kind 1 (amplitudes): outT[g][t][lane] = sqrt(w_t) dout[inst][t]   (complex)
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
            uint32_t supp = 0;
            float fp = 1.f;
#pragma unroll
            for (int j = 0; j < MMAX; ++j) {
                if (j < m) {
                    const int tj = occupation<MMAX>(j, m, L, p);
                    fp *= c_fact.v[tj];
                    if (tj > 0) supp |= 1u << j;
                }
            }
            const float w = fp * a.inv_sfact;
            int64_t idx = c;
            if (a.kind == 2) idx = a.pat_off[__popc(supp)] + (int64_t)colex_rank(supp);
            const int64_t src = (valid ? (int64_t)inst * a.stride : 0) + idx;
            if (a.kind == 1) {
                float2 v = valid ? __ldg(reinterpret_cast<const float2 *>(a.dout) + src) : make_float2(0.f, 0.f);
                reinterpret_cast<float2 *>(a.outT)[(base + c) * kLanes + lane] = cscale(v, sqrtf(w));
            } else {
                float v = valid ? __ldg(reinterpret_cast<const float *>(a.dout) + src) : 0.f;
                reinterpret_cast<float *>(a.outT)[(base + c) * kLanes + lane] = 2.f * w * v;
            }
            next_bars<MMAX>(m, L, p);
        }
    }
}

// Shared seed (dout row stride 0): dpw[t] = 2 w_t dout[t] (PNR) or
// 2 w_t dout[pattern(t)] (threshold); one thread per state.
template <int MMAX>
__global__ void slos_seed_bcast_kernel(PrepArgs a) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.Fn) return;
    const int m = a.m;
    const int L = a.n + m - 1;
    int p[MMAX];
    unrank_bars<MMAX>(c, m, L, p);
    uint32_t supp = 0;
    float fp = 1.f;
#pragma unroll
    for (int j = 0; j < MMAX; ++j) {
        if (j < m) {
            const int tj = occupation<MMAX>(j, m, L, p);
            fp *= c_fact.v[tj];
            if (tj > 0) supp |= 1u << j;
        }
    }
    int64_t idx = c;
    if (a.kind == 2) idx = a.pat_off[__popc(supp)] + (int64_t)colex_rank(supp);
    reinterpret_cast<float *>(a.outT)[c] = 2.f * fp * a.inv_sfact * __ldg(reinterpret_cast<const float *>(a.dout) + idx);
}

// ------------------------------------------------------------------ table mode
// Backward with the precomputed child table: per parent, lane j < m fetches
// rank_k(t' + e_j); the warp broadcasts each child index and gathers the child
// gradients with independent coalesced loads, 8 modes at a time.  U[j, c_k]
// lives in shared memory and only dU stays in registers.
//
// Register budget (resident 4-warp blocks per SM): the final layer, which
// also forms the child gradient from a_n and the seed, runs fastest at 64
// registers (8 blocks, a few bytes of spill) for up to 16 modes; the
// intermediate layers at about 80 (6 blocks).  Plans of 13-16 modes use
// slos_bwd_tmem_kernel below instead, whose dU accumulators live in tensor
// memory.
constexpr int kBwdTabWarps = 4;
constexpr int kBwdTabBatch = 8;  // child gathers issued together per parent
// final layer of 16-mode plans, dU in tensor memory: 9 blocks (56 registers,
// no spill) measured 0.890 ms per step against 1.077 ms with the register
// accumulators at 8; 8 blocks the same, 10 (spills) 0.960 ms
constexpr int kBwdTmemMinBlocks = 9;
constexpr int kBwdTmemLayerMinBlocks = 8;  // the other layers of 16-mode plans: 0.472 -> 0.430 ms (9 blocks 0.435)
constexpr int bwd_tab_min_blocks(int mmax, bool final_layer) {
    return final_layer ? (mmax == 16 ? kBwdTmemMinBlocks : (mmax < 16 ? 8 : 6)) : (mmax == 16 ? kBwdTmemLayerMinBlocks : 6);
}


// HOLES: the child table may name no child (-1), for lattices where t' + e_j
// leaves the space (collision-free states); such children contribute nothing.
template <int MMAX, int SEED, int MINB, bool HOLES, int BATCH = kBwdTabBatch>
__global__ void __launch_bounds__(kBwdTabWarps * 32, MINB) slos_bwd_tab_kernel(BwdArgs a, const int32_t *ctab) {
    __shared__ float2 red[kBwdTabWarps][32];
    __shared__ float2 us[MMAX][32];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int grp = blockIdx.y;
    const int inst = grp * kLanes + lane;
    const bool valid = inst < a.B;
    const int m = a.m;
    for (int j = warp; j < m; j += kBwdTabWarps)
        us[j][lane] = valid ? a.U[((int64_t)inst * m + j) * m + a.col] : make_float2(0.f, 0.f);
    __syncthreads();
    float2 dU[MMAX];
#pragma unroll
    for (int j = 0; j < MMAX; ++j) dU[j] = make_float2(0.f, 0.f);
    // 64-bit group bases once; per-state offsets are 32-bit (table plans: F * 32 < 2^32)
    const size_t gprev = (size_t)grp * (size_t)a.Fprev * kLanes + lane;
    const size_t gk = (size_t)grp * (size_t)a.Fk * kLanes + lane;
    const float2 *aprevb = a.aprev + gprev;
    float2 *Gprevb = a.Gprev + gprev;
    // child gradient source: G_k, or a_n with a per-instance / shared seed
    const float2 *srcb = (SEED == SEED_G) ? a.Gk + gk
                         : (SEED == SEED_AMPS_T) ? reinterpret_cast<const float2 *>(a.seed) + gk : a.an + gk;
    const float *seedb = (SEED == SEED_T) ? reinterpret_cast<const float *>(a.seed) + gk
                                          : reinterpret_cast<const float *>(a.seed);
    const uint32_t nwarps = gridDim.x * kBwdTabWarps;
    for (uint32_t c = blockIdx.x * kBwdTabWarps + warp; c < (uint32_t)a.Fprev; c += nwarps) {
        const int mine = lane < m ? __ldg(ctab + (size_t)c * m + lane) : 0;
        const float2 av = (a.k == 1) ? make_float2(1.f, 0.f) : __ldg(aprevb + (c << 5));
        float2 gacc = make_float2(0.f, 0.f);
#pragma unroll
        for (int h = 0; h < MMAX; h += BATCH) {
            float2 g[BATCH];
#pragma unroll
            for (int r = 0; r < BATCH; ++r) {
                const int j = h + r;
                const uint32_t cidx = (uint32_t)__shfl_sync(0xffffffffu, mine, j < 32 ? j : 0);
                g[r] = make_float2(0.f, 0.f);
                if (j < m && (!HOLES || (int)cidx >= 0)) {
                    g[r] = __ldg(srcb + (cidx << 5));
                    if (SEED == SEED_T) g[r] = cscale(g[r], __ldg(seedb + (cidx << 5)));
                    if (SEED == SEED_BCAST) g[r] = cscale(g[r], __ldg(seedb + cidx));
                }
            }
#pragma unroll
            for (int r = 0; r < BATCH; ++r) {
                const int j = h + r;
                if (j < MMAX && j < m) {
                    gacc = cfma_conj_a(us[j][lane], g[r], gacc);
                    dU[j] = cfma_conj_a(av, g[r], dU[j]);
                }
            }
        }
        if (a.k > 1) Gprevb[c << 5] = gacc;
    }
    float2 *dst = a.dUpart + (((int64_t)grp * gridDim.x + blockIdx.x) * kLanes) * m;
#pragma unroll
    for (int j = 0; j < MMAX; ++j) {
        if (j < m) {
            red[warp][lane] = dU[j];
            __syncthreads();
            if (warp == 0) {
                float2 sacc = red[0][lane];
#pragma unroll
                for (int w = 1; w < kBwdTabWarps; ++w) {
                    sacc.x += red[w][lane].x;
                    sacc.y += red[w][lane].y;
                }
                dst[lane * m + j] = sacc;
            }
            __syncthreads();
        }
    }
}

// Tensor-memory accumulators.  Each warp of a CTA owns one 32-lane quarter
// of the CTA's tensor memory (warp w: lanes 32 w .. 32 w + 31); 32x32b
// loads and stores move 16 consecutive 32-bit columns of that quarter
// between TMEM and 16 registers per lane.
__device__ __forceinline__ void tm_ld16(uint32_t taddr, float (&v)[16]) {
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
__device__ __forceinline__ void tm_st16(uint32_t taddr, const float (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
        "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
        "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Final backward layer of 16-mode plans with the dU accumulators in tensor
// memory instead of registers: per batch of 8 modes a warp loads its 8
// accumulators (16 columns), adds conj(a_{k-1}) G_k for the batch's children
// and stores them back, so only 8 of the 16 live in registers at a time and
// the register budget admits more resident warps.  TMEM traffic has its own
// datapath, not the L1 / shared-memory pipe the gathers use.  32 columns per
// CTA (the minimum allocation); the CTA frees them before it exits.
constexpr int kBwdTmemCols = 32;
template <int MMAX, int SEED, int MINB, bool HOLES>
__global__ void __launch_bounds__(kBwdTabWarps * 32, MINB) slos_bwd_tmem_kernel(BwdArgs a, const int32_t *ctab) {
    static_assert(MMAX == 16 && kBwdTabBatch == 8, "two batches of 8 modes, 32 TMEM columns");
    __shared__ float2 red[kBwdTabWarps][32];
    __shared__ float2 us[MMAX][32];
    __shared__ uint32_t tmem_slot;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int grp = blockIdx.y;
    const int inst = grp * kLanes + lane;
    const bool valid = inst < a.B;
    const int m = a.m;
    for (int j = warp; j < m; j += kBwdTabWarps)
        us[j][lane] = valid ? a.U[((int64_t)inst * m + j) * m + a.col] : make_float2(0.f, 0.f);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         static_cast<uint32_t>(__cvta_generic_to_shared(&tmem_slot))),
                     "r"(kBwdTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tq = tmem_slot + ((uint32_t)(warp * 32) << 16);  // this warp's lane quarter
    {
        float z[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) z[i] = 0.f;
        tm_st16(tq, z);
        tm_st16(tq + 16, z);
    }
    const size_t gprev = (size_t)grp * (size_t)a.Fprev * kLanes + lane;
    const size_t gk = (size_t)grp * (size_t)a.Fk * kLanes + lane;
    const float2 *aprevb = a.aprev + gprev;
    float2 *Gprevb = a.Gprev + gprev;
    const float2 *srcb = (SEED == SEED_G) ? a.Gk + gk
                         : (SEED == SEED_AMPS_T) ? reinterpret_cast<const float2 *>(a.seed) + gk : a.an + gk;
    const float *seedb = (SEED == SEED_T) ? reinterpret_cast<const float *>(a.seed) + gk
                                          : reinterpret_cast<const float *>(a.seed);
    const uint32_t nwarps = gridDim.x * kBwdTabWarps;
    for (uint32_t c = blockIdx.x * kBwdTabWarps + warp; c < (uint32_t)a.Fprev; c += nwarps) {
        const int mine = lane < m ? __ldg(ctab + (size_t)c * m + lane) : 0;
        const float2 av = (a.k == 1) ? make_float2(1.f, 0.f) : __ldg(aprevb + (c << 5));
        float2 gacc = make_float2(0.f, 0.f);
#pragma unroll
        for (int h = 0; h < MMAX; h += 8) {
            float2 g[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int j = h + r;
                const uint32_t cidx = (uint32_t)__shfl_sync(0xffffffffu, mine, j);
                g[r] = make_float2(0.f, 0.f);
                if (j < m && (!HOLES || (int)cidx >= 0)) {
                    g[r] = __ldg(srcb + (cidx << 5));
                    if (SEED == SEED_T) g[r] = cscale(g[r], __ldg(seedb + (cidx << 5)));
                    if (SEED == SEED_BCAST) g[r] = cscale(g[r], __ldg(seedb + cidx));
                }
            }
            float du[16];
            tm_ld16(tq + 2 * h, du);
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int j = h + r;
                if (j < m) {
                    gacc = cfma_conj_a(us[j][lane], g[r], gacc);
                    const float2 d = cfma_conj_a(av, g[r], make_float2(du[2 * r], du[2 * r + 1]));
                    du[2 * r] = d.x;
                    du[2 * r + 1] = d.y;
                }
            }
            tm_st16(tq + 2 * h, du);
        }
        if (a.k > 1) Gprevb[c << 5] = gacc;
    }
    float2 *dst = a.dUpart + (((int64_t)grp * gridDim.x + blockIdx.x) * kLanes) * m;
#pragma unroll
    for (int h = 0; h < MMAX; h += 8) {
        float du[16];
        tm_ld16(tq + 2 * h, du);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int j = h + r;
            if (j < m) {
                red[warp][lane] = make_float2(du[2 * r], du[2 * r + 1]);
                __syncthreads();
                if (warp == 0) {
                    float2 sacc = red[0][lane];
#pragma unroll
                    for (int w = 1; w < kBwdTabWarps; ++w) {
                        sacc.x += red[w][lane].x;
                        sacc.y += red[w][lane].y;
                    }
                    dst[lane * m + j] = sacc;
                }
                __syncthreads();
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_slot), "r"(kBwdTmemCols)
                     : "memory");
    }
}

// ------------------------------------------------------------------ launchers
inline size_t fwd_smem_bytes(int epi) {
    if (epi == EPI_PROBS) return (size_t)kWarpsPerBlock * 32 * 33 * sizeof(float);
    if (epi == EPI_AMPS) return (size_t)kWarpsPerBlock * 32 * 33 * sizeof(float2);
    return 0;
}

template <int MM, bool HOLES>
cudaError_t launch_bwd_tab_t(const BwdArgs &a, const int32_t *ctab, int seed, int blocks_x, cudaStream_t s) {
    dim3 grid(blocks_x, a.NG);
    constexpr int mg = bwd_tab_min_blocks(MM, false), mf = bwd_tab_min_blocks(MM, true);
    switch (seed) {
        case SEED_G:
            if constexpr (MM == 16) slos_bwd_tmem_kernel<16, SEED_G, mg, HOLES><<<grid, kBwdTabWarps * 32, 0, s>>>(a, ctab);
            else slos_bwd_tab_kernel<MM, SEED_G, mg, HOLES><<<grid, kBwdTabWarps * 32, 0, s>>>(a, ctab);
            break;
        case SEED_BCAST:
            if constexpr (MM == 16) slos_bwd_tmem_kernel<16, SEED_BCAST, mf, HOLES><<<grid, kBwdTabWarps * 32, 0, s>>>(a, ctab);
            else slos_bwd_tab_kernel<MM, SEED_BCAST, mf, HOLES><<<grid, kBwdTabWarps * 32, 0, s>>>(a, ctab);
            break;
        case SEED_T:
            if constexpr (MM == 16) slos_bwd_tmem_kernel<16, SEED_T, mf, HOLES><<<grid, kBwdTabWarps * 32, 0, s>>>(a, ctab);
            else slos_bwd_tab_kernel<MM, SEED_T, mf, HOLES><<<grid, kBwdTabWarps * 32, 0, s>>>(a, ctab);
            break;
        case SEED_AMPS_T:
            if constexpr (MM == 16) slos_bwd_tmem_kernel<16, SEED_AMPS_T, mf, HOLES><<<grid, kBwdTabWarps * 32, 0, s>>>(a, ctab);
            else slos_bwd_tab_kernel<MM, SEED_AMPS_T, mf, HOLES><<<grid, kBwdTabWarps * 32, 0, s>>>(a, ctab);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Defines the host launchers of one MMAX instantiation (one per .cu file so
// the instantiations compile in parallel).
#define SLOS_DEFINE_LAUNCHERS(MM)                                                                            \
    cudaError_t slos_init_m##MM() {                                                                          \
        const int sm = (int)fwd_smem_bytes(EPI_AMPS);                                                        \
        cudaError_t e = cudaFuncSetAttribute(slos_fwd_kernel<MM, EPI_AMPS, false, kCFinal>,                          \
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, sm);               \
        if (e != cudaSuccess) return e;                                                                      \
        return cudaFuncSetAttribute(slos_fwd_kernel<MM, EPI_AMPS, true, kCFinal>,                                    \
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, sm);                        \
    }                                                                                                        \
    cudaError_t slos_launch_fwd_m##MM(const FwdArgs &a, int epi, bool save, int blocks_x, cudaStream_t s) { \
        dim3 grid(blocks_x, a.NG);                                                                           \
        const size_t sm = fwd_smem_bytes(epi);                                                               \
        switch (epi * 2 + (save ? 1 : 0)) {                                                                  \
            case 0:                                                                                          \
            case 1: slos_fwd_kernel<MM, EPI_STORE, true, kCStore><<<grid, kThreads, 0, s>>>(a); break;               \
            case 2: slos_fwd_kernel<MM, EPI_PROBS, false, kCFinal><<<grid, kThreads, sm, s>>>(a); break;             \
            case 3: slos_fwd_kernel<MM, EPI_PROBS, true, kCFinal><<<grid, kThreads, sm, s>>>(a); break;              \
            case 4: slos_fwd_kernel<MM, EPI_AMPS, false, kCFinal><<<grid, kThreads, sm, s>>>(a); break;              \
            case 5: slos_fwd_kernel<MM, EPI_AMPS, true, kCFinal><<<grid, kThreads, sm, s>>>(a); break;               \
            default: return cudaErrorInvalidValue;                                                           \
        }                                                                                                    \
        return cudaGetLastError();                                                                           \
    }                                                                                                        \
    cudaError_t slos_launch_bwd_m##MM(const BwdArgs &a, int seed, int blocks_x, cudaStream_t s) {           \
        dim3 grid(blocks_x, a.NG);                                                                           \
        switch (seed) {                                                                                      \
            case SEED_G: slos_bwd_kernel<MM, SEED_G, kCBwd><<<grid, kThreads, 0, s>>>(a); break;                   \
            case SEED_BCAST: slos_bwd_kernel<MM, SEED_BCAST, kCBwd><<<grid, kThreads, 0, s>>>(a); break;             \
            case SEED_T: slos_bwd_kernel<MM, SEED_T, kCBwd><<<grid, kThreads, 0, s>>>(a); break;                     \
            case SEED_AMPS_T: slos_bwd_kernel<MM, SEED_AMPS_T, kCBwd><<<grid, kThreads, 0, s>>>(a); break;         \
            default: return cudaErrorInvalidValue;                                                           \
        }                                                                                                    \
        return cudaGetLastError();                                                                           \
    }                                                                                                        \
    cudaError_t slos_launch_prep_m##MM(const PrepArgs &a, int blocks_x, bool bcast, cudaStream_t s) {       \
        if (bcast) {                                                                                         \
            slos_seed_bcast_kernel<MM><<<(unsigned)((a.Fn + 255) / 256), 256, 0, s>>>(a);                    \
        } else {                                                                                             \
            dim3 grid(blocks_x, a.NG);                                                                       \
            slos_seed_prep_kernel<MM><<<grid, kThreads, 0, s>>>(a);                                          \
        }                                                                                                    \
        return cudaGetLastError();                                                                           \
    }                                                                                                        \
    cudaError_t slos_launch_bwd_tab_m##MM(const BwdArgs &a, const int32_t *ctab, int seed, int blocks_x,    \
                                          bool holes, cudaStream_t s) {                                      \
        return holes ? launch_bwd_tab_t<MM, true>(a, ctab, seed, blocks_x, s)                                \
                     : launch_bwd_tab_t<MM, false>(a, ctab, seed, blocks_x, s);                              \
    }

#define SLOS_DECLARE_LAUNCHERS(MM)                                                                  \
    cudaError_t slos_init_m##MM();                                                                  \
    cudaError_t slos_launch_fwd_m##MM(const FwdArgs &a, int epi, bool save, int blocks_x, cudaStream_t s); \
    cudaError_t slos_launch_bwd_m##MM(const BwdArgs &a, int seed, int blocks_x, cudaStream_t s);  \
    cudaError_t slos_launch_prep_m##MM(const PrepArgs &a, int blocks_x, bool bcast, cudaStream_t s);      \
    cudaError_t slos_launch_bwd_tab_m##MM(const BwdArgs &a, const int32_t *ctab, int seed, int blocks_x,  \
                                          bool holes, cudaStream_t s);

}  // namespace slos
