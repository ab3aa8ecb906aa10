// SLOS layers on the head/tail split of the Fock lattice (split.h).
//
// The forward layers do not use the split: a head-block walk that takes
// the head parents at fixed offsets measured slower on GB300 than the
// two-group slot-table walk of slos_pair.cu, whose slot rows are shared by
// both instance groups of a warp.
//
// Backward, layer k:  for every parent t' of layer k-1
//      G_{k-1}(t') = sum_j conj(U[j, c_k]) G_k(t' + e_j)
//      dU[j, c_k] += conj(a_{k-1}(t')) G_k(t' + e_j)
// with all m children present: head children at fixed offsets per block,
// tail children from the tail child row.  The mode of every child is a
// compile-time index, so U[j, c_k] and the dU accumulators sit in tensor
// memory (one 32-lane quarter per warp, 16 columns per batch of 8 modes) and
// move with one tcgen05.ld / tcgen05.st per batch instead of per-child
// shared-memory loads.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "slos_kernels.cuh"
#include "split.h"
#include "tab_launch.h"

namespace slos {

// ============================================================ host tables
int64_t binom_host(int a, int e);
int64_t host_rank(int m, const int *t);

// Successor in descending lexicographic order among compositions with the
// same sum; false after the last one, (0, ..., 0, sum).
static bool next_comp_desc(std::vector<int> &t) {
    const int P = (int)t.size();
    int i = P - 2;
    while (i >= 0 && t[i] == 0) --i;
    if (i < 0) return false;
    int rest = 0;
    for (int q = i + 1; q < P; ++q) {
        rest += t[q];
        t[q] = 0;
    }
    t[i] -= 1;
    t[i + 1] = rest + 1;
    return true;
}

bool split_eligible(int m, int n, int *h_out) {
    if (m < 8 || m > 16 || n < 2) return false;
    const int h = m >= 13 ? 8 : 6;
    const int mL = m - h;
    if (mL < 1 || mL > kSplitMaxTail || h > kSplitMaxHead) return false;
    if (binom_host(n + mL - 1, n) > kSplitMaxTailStates) return false;
    if (h_out) *h_out = h;
    return true;
}

void split_build_layer_host(int m, int h, int k, SplitLayerHost &out) {
    const int mL = m - h;
    std::vector<int> full(m, 0);
    // backward: head compositions of at most k-1 photons (the parents)
    {
        out.bdesc.clear();
        out.bhead.clear();
        std::vector<int> tc(h + 1, 0);
        tc[0] = k - 1;
        do {
            const int rho = tc[h];
            std::fill(full.begin(), full.end(), 0);
            for (int j = 0; j < h; ++j) full[j] = tc[j];
            full[h] = rho;
            const int64_t base = host_rank(m, full.data());
            const int64_t size = binom_host(rho + mL - 1, mL - 1);
            full[h] = rho + 1;
            const int64_t lcb = host_rank(m, full.data());
            full[h] = rho;
            out.bdesc.push_back((int32_t)base);
            out.bdesc.push_back((int32_t)size);
            out.bdesc.push_back((int32_t)lcb);
            out.bdesc.push_back(rho);
            for (int j = 0; j < kSplitMaxHead; ++j) {
                if (j < h) {
                    full[j] += 1;
                    out.bhead.push_back((int32_t)host_rank(m, full.data()));
                    full[j] -= 1;
                } else {
                    out.bhead.push_back(0);
                }
            }
        } while (next_comp_desc(tc));
        const int64_t Fp = binom_host(m + k - 2, k - 1);
        out.bchunk.assign((size_t)((Fp + kSplitRun - 1) / kSplitRun), 0);
        const size_t nb = out.bdesc.size() / 4;
        for (size_t b = 0; b < nb; ++b) {
            const int64_t lo = out.bdesc[4 * b], hi = lo + out.bdesc[4 * b + 1];
            for (int64_t c0 = (lo + kSplitRun - 1) / kSplitRun * kSplitRun; c0 < hi; c0 += kSplitRun)
                out.bchunk[(size_t)(c0 / kSplitRun)] = (int32_t)b;
        }
    }
}

void split_build_tail_host(int m, int h, int n, SplitTailHost &out) {
    const int mL = m - h;
    out.ctab.clear();
    std::vector<int> t(mL, 0);
    for (int rho = 0; rho <= n; ++rho) {
        out.coff[rho] = (int)(out.ctab.size() / 8);
        if (rho == n) break;  // the last layer's states have no children
        std::fill(t.begin(), t.end(), 0);
        t[0] = rho;
        do {
            for (int j = 0; j < 8; ++j) {
                uint16_t v = 0;
                if (j < mL) {
                    t[j] += 1;
                    v = (uint16_t)host_rank(mL, t.data());
                    t[j] -= 1;
                }
                out.ctab.push_back(v);
            }
        } while (mL > 1 && next_comp_desc(t));
    }
}

// ============================================================ backward kernel
// 8-column tensor-memory moves (4 complex values per lane).  The wait on the
// loads names the loaded registers, so no use of them can be scheduled
// before it; none of these statements is a compiler memory barrier, so the
// global loads of the children stay free to move around them.
__device__ __forceinline__ void tm_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}
__device__ __forceinline__ void tm_wait_ld8(uint32_t (&r)[8], uint32_t (&q)[8]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(q[0]), "+r"(q[1]), "+r"(q[2]), "+r"(q[3]), "+r"(q[4]), "+r"(q[5]), "+r"(q[6]), "+r"(q[7]));
}
__device__ __forceinline__ void tm_st8(uint32_t taddr, const uint32_t (&r)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]));
    asm volatile("tcgen05.wait::st.sync.aligned;");
}

// 16-bit local child position J of a tail child row
template <int J>
__device__ __forceinline__ uint32_t crow16(const uint4 &r) {
    const uint32_t w = J < 2 ? r.x : (J < 4 ? r.y : (J < 6 ? r.z : r.w));
    return (J & 1) ? (w >> 16) : (w & 0xffffu);
}

template <int SEED>
__device__ __forceinline__ float2 split_child(const float2 *srcb, const float *seedb, uint32_t x, uint32_t fk,
                                              int *status) {
    (void)fk;
    (void)status;
    x = SLOS_IDX(x, fk, status);
    float2 g = __ldg(srcb + (x << 5));
    if (SEED == SEED_T) g = cscale(g, __ldg(seedb + (x << 5)));
    if (SEED == SEED_BCAST) g = cscale(g, __ldg(seedb + x));
    return g;
}

// The same for a runtime q.
__device__ __forceinline__ uint32_t crow16_rt(const uint4 &r, int q) {
    const uint32_t w = q < 2 ? r.x : (q < 4 ? r.y : (q < 6 ? r.z : r.w));
    return (q & 1) ? (w >> 16) : (w & 0xffffu);
}

// Tail child J of a parent (local position from the tail child row), 0 past
// the plan's tail modes.
template <int J, int SEED>
__device__ __forceinline__ float2 tail_child(const float2 *srcb, const float *seedb, uint32_t lc, const uint4 &cr,
                                             int mL, uint32_t fk, int *status) {
    return mL > J ? split_child<SEED>(srcb, seedb, lc + crow16<J>(cr), fk, status) : make_float2(0.f, 0.f);
}

// One batch of (up to) 4 children of a parent: G_{k-1} += conj(U_j) g_j and
// dU_j += conj(a_{k-1}) g_j, with dU_j and U_j in tensor-memory columns
// [cd, cd + 8) and [cu, cu + 8) of the warp's lane quarter.  Modes past the
// plan's last one hold U = 0 and g = 0.
template <int N>
__device__ __forceinline__ void split_bwd_batch(uint32_t tq, uint32_t cd, uint32_t cu, const float2 *g, float2 av,
                                                float2 &gacc) {
    uint32_t du[8], uu[8];
    tm_ld8(tq + cd, du);
    tm_ld8(tq + cu, uu);
    tm_wait_ld8(du, uu);
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const float2 u = make_float2(__uint_as_float(uu[2 * j]), __uint_as_float(uu[2 * j + 1]));
        gacc = cfma_conj_a(u, g[j], gacc);
        const float2 d = cfma_conj_a(av, g[j], make_float2(__uint_as_float(du[2 * j]), __uint_as_float(du[2 * j + 1])));
        du[2 * j] = __float_as_uint(d.x);
        du[2 * j + 1] = __float_as_uint(d.y);
    }
    tm_st8(tq + cd, du);
}

// TMEM columns of a warp's lane quarter: dU of the head modes [0, 16), of the
// tail modes [16, 32); U[j, c_k] of the head modes [32, 48), tail [48, 64).
constexpr int kSplitTmemCols = 64;

template <int H, int SEED, bool FUSE = false>
__global__ void __launch_bounds__(kSplitBwdWarps * 32, kSplitBwdMinBlocks) slos_bwd_split_kernel(SplitBwdArgs a) {
    constexpr int T = kSplitMaxTail;
    __shared__ float2 red[kSplitBwdWarps][32];
    // FUSE: U[j, c_{k-1}] of the group's instances, row kMaxModes zero (padding slots)
    __shared__ float2 upc[FUSE ? kMaxModes + 1 : 1][32];
    __shared__ uint32_t tmem_slot;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int grp = blockIdx.y;
    const int inst = grp * kLanes + lane;
    const bool valid = inst < a.B;
    const int m = a.m;
    const int mL = m - H;
    if (FUSE && warp == 1) {
        for (int j = 0; j <= kMaxModes; ++j)
            upc[j][lane] = (valid && j < m) ? a.U[((int64_t)inst * m + j) * m + a.pcol] : make_float2(0.f, 0.f);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         static_cast<uint32_t>(__cvta_generic_to_shared(&tmem_slot))),
                     "r"(kSplitTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tq = tmem_slot + ((uint32_t)(warp * 32) << 16);
    {
        float z[16], uh[16], ut[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) z[i] = 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float2 u = make_float2(0.f, 0.f), v = make_float2(0.f, 0.f);
            if (valid && j < H) u = a.U[((int64_t)inst * m + j) * m + a.col];
            if (valid && j < mL) v = a.U[((int64_t)inst * m + H + j) * m + a.col];
            uh[2 * j] = u.x;
            uh[2 * j + 1] = u.y;
            ut[2 * j] = v.x;
            ut[2 * j + 1] = v.y;
        }
        tm_st16(tq, z);
        tm_st16(tq + 16, z);
        tm_st16(tq + 32, uh);
        tm_st16(tq + 48, ut);
    }
    const size_t gprev = (size_t)grp * (size_t)a.Fprev * kLanes + lane;
    const size_t gk = (size_t)grp * (size_t)a.Fk * kLanes + lane;
    const float2 *aprevb = a.aprev + gprev;
    const float2 *pprevb = FUSE ? a.pprev + (size_t)grp * (size_t)a.Fpp * kLanes + lane : nullptr;
    float2 *Gprevb = a.Gprev + gprev;
    const float2 *srcb = (SEED == SEED_G) ? a.Gk + gk
                         : (SEED == SEED_AMPS_T) ? reinterpret_cast<const float2 *>(a.seed) + gk : a.an + gk;
    const float *seedb = (SEED == SEED_T) ? reinterpret_cast<const float *>(a.seed) + gk
                                          : reinterpret_cast<const float *>(a.seed);
    const int wstride = gridDim.x * kSplitBwdWarps;
    const uint32_t fk = (uint32_t)a.Fk;
    int *const st = a.status;
    const float2 z = make_float2(0.f, 0.f);
    for (int ch = blockIdx.x * kSplitBwdWarps + warp; ch < a.nruns; ch += wstride) {
        const int c0 = ch * kSplitRun;
        const int cend = min(c0 + kSplitRun, a.Fprev);
        int b = __ldg(a.chunk + ch);
        for (int c = c0; c < cend; ++b) {
            const int4 d = __ldg(reinterpret_cast<const int4 *>(a.desc) + b);
            const int stop = min(d.x + d.y, cend);
            int hoff[8];
            {
                const int4 h0 = __ldg(reinterpret_cast<const int4 *>(a.head) + 2 * b);
                const int4 h1 = __ldg(reinterpret_cast<const int4 *>(a.head) + 2 * b + 1);
                const int hv[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
#pragma unroll
                for (int j = 0; j < 8; ++j) hoff[j] = hv[j] - d.x;  // head child of parent c: c + hoff[j]
            }
            const uint4 *crow = reinterpret_cast<const uint4 *>(a.tctab) + a.coff[d.w] + (c - d.x);
            const uint32_t lc = (uint32_t)d.z;
            for (; c < stop; ++c, ++crow) {
                float2 av;
                if (FUSE) {
                    // a_{k-1}(c) = sum over its parent slots of U[j, c_{k-1}] a_{k-2}(parent)
                    const uint4 *sr = reinterpret_cast<const uint4 *>(a.pslots) + (size_t)c * 2;
                    const uint4 s0 = __ldg(sr), s1 = __ldg(sr + 1);
                    const uint32_t e[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
                    av = make_float2(0.f, 0.f);
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        av = cfma(upc[e[q] & 31u][lane], __ldg(pprevb + ((e[q] >> 5) << 5)), av);
                } else {
                    av = __ldg(aprevb + ((uint32_t)c << 5));
                }
                const uint4 cr = __ldg(crow);
                float2 gacc = make_float2(0.f, 0.f);
                // every child of the parent first (16 loads in flight), then the four
                // tensor-memory batches: head modes 0..3, 4..H-1, tail modes 0..3, 4..7
                float2 g[16];
#pragma unroll
                for (int j = 0; j < 8; ++j) g[j] = j < H ? split_child<SEED>(srcb, seedb, c + hoff[j], fk, st) : z;
                g[8] = tail_child<0, SEED>(srcb, seedb, lc, cr, mL, fk, st);
                g[9] = tail_child<1, SEED>(srcb, seedb, lc, cr, mL, fk, st);
                g[10] = tail_child<2, SEED>(srcb, seedb, lc, cr, mL, fk, st);
                g[11] = tail_child<3, SEED>(srcb, seedb, lc, cr, mL, fk, st);
                g[12] = tail_child<4, SEED>(srcb, seedb, lc, cr, mL, fk, st);
                g[13] = tail_child<5, SEED>(srcb, seedb, lc, cr, mL, fk, st);
                g[14] = tail_child<6, SEED>(srcb, seedb, lc, cr, mL, fk, st);
                g[15] = tail_child<7, SEED>(srcb, seedb, lc, cr, mL, fk, st);
                split_bwd_batch<4>(tq, 0, 32, g, av, gacc);
                split_bwd_batch<H - 4>(tq, 8, 40, g + 4, av, gacc);
                split_bwd_batch<4>(tq, 16, 48, g + 8, av, gacc);
                split_bwd_batch<4>(tq, 24, 56, g + 12, av, gacc);
                Gprevb[(uint32_t)c << 5] = gacc;
            }
        }
    }
    static_assert(T == 8, "two tail batches of 4 modes");
    // reduce dU over the CTA's warps, one mode at a time
    float2 *dst = a.dUpart + (((int64_t)grp * gridDim.x + blockIdx.x) * kLanes) * m;
    {
        float dh[16], dt[16];
        tm_ld16(tq, dh);
        tm_ld16(tq + 16, dt);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (j < m) {
                red[warp][lane] = j < H ? make_float2(dh[2 * j], dh[2 * j + 1])
                                        : make_float2(dt[2 * (j - H)], dt[2 * (j - H) + 1]);
                __syncthreads();
                if (warp == 0) {
                    float2 s = red[0][lane];
#pragma unroll
                    for (int w = 1; w < kSplitBwdWarps; ++w) {
                        s.x += red[w][lane].x;
                        s.y += red[w][lane].y;
                    }
                    dst[lane * m + j] = s;
                }
                __syncthreads();
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_slot), "r"(kSplitTmemCols)
                     : "memory");
    }
}

// ============================================================ ring kernel
// The final layer (seed rows a_n or the amplitude seed) with each parent's
// rows staged through a per-warp ring of kRingDepth shared-memory stages
// filled by cp.async: while a warp sums one parent, the 16 child rows, the
// parent row and (batch-shared seed) the 16 seeds of the next parent are in
// flight without holding registers.  Rows move in 16-byte copies that skip
// L1 (a half-warp per row), so every lane reads its own instance of each row
// after a __syncwarp; the seeds are fetched by lanes 0..15.  Measured on GB300 (m=16, n=8, batch 256): final layer 0.785 ->
// 0.715 ms; the intermediate layers, whose child rows G_k mostly hit L2, ran
// slower this way (0.326 -> 0.355 ms) and keep the register walk above.
constexpr int kRingDepth = 2;
constexpr int kRingRows = 18;                       // children 0..15, parent row, seeds
constexpr int kRingStage = kRingRows * kLanes * 8;  // bytes per stage
constexpr int kRingWarpBytes = kRingDepth * kRingStage;
size_t split_ring_smem_bytes() { return (size_t)kSplitBwdWarps * kRingWarpBytes; }

__device__ __forceinline__ void cp_async8(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// The issue cursor of a warp: runs of kSplitRun parents (ch, ch + stride, ...),
// crossing head blocks where they must, with the head offsets of the block.
struct RingCursor {
    int ch, c, cend, stop, b;
    int4 d;
    const uint4 *crow;
    int hoff[8];
    int hl;  // lane l < 8: the head offset of mode l (for its seed)
};
__device__ __forceinline__ void ring_block(RingCursor &w, const SplitBwdArgs &a, int lane) {
    w.d = __ldg(reinterpret_cast<const int4 *>(a.desc) + w.b);
    w.stop = min(w.d.x + w.d.y, w.cend);
    w.crow = reinterpret_cast<const uint4 *>(a.tctab) + a.coff[w.d.w] + (w.c - w.d.x);
    const int4 h0 = __ldg(reinterpret_cast<const int4 *>(a.head) + 2 * w.b);
    const int4 h1 = __ldg(reinterpret_cast<const int4 *>(a.head) + 2 * w.b + 1);
    w.hoff[0] = h0.x - w.d.x;
    w.hoff[1] = h0.y - w.d.x;
    w.hoff[2] = h0.z - w.d.x;
    w.hoff[3] = h0.w - w.d.x;
    w.hoff[4] = h1.x - w.d.x;
    w.hoff[5] = h1.y - w.d.x;
    w.hoff[6] = h1.z - w.d.x;
    w.hoff[7] = h1.w - w.d.x;
    w.hl = __ldg(a.head + 8 * w.b + (lane & 7)) - w.d.x;
}
__device__ __forceinline__ bool ring_run(RingCursor &w, const SplitBwdArgs &a, int lane) {
    if (w.ch >= a.nruns) return false;
    w.c = w.ch * kSplitRun;
    w.cend = min(w.c + kSplitRun, a.Fprev);
    w.b = __ldg(a.chunk + w.ch);
    ring_block(w, a, lane);
    return true;
}
__device__ __forceinline__ bool ring_next(RingCursor &w, const SplitBwdArgs &a, int stride, int lane) {
    ++w.c;
    ++w.crow;
    if (w.c >= w.cend) {
        w.ch += stride;
        return ring_run(w, a, lane);
    }
    if (w.c >= w.stop) {
        ++w.b;
        ring_block(w, a, lane);
    }
    return true;
}

// Copies of parent w.c into a stage (one commit group, possibly empty): each
// 16-byte copy (L2 only) moves 4 instances, so a half-warp moves a 256-byte
// row and the warp two rows per instruction: rows 2i (lanes 0..15) and 2i + 1
// (lanes 16..31).  Rows of modes past the plan's are never copied.
template <int H, int SEED>
__device__ __forceinline__ void ring_issue(const RingCursor &w, const uint4 &cr, uint32_t stage, int lane, int mL,
                                           const char *srcg, const char *aprevg, const float *seedb, uint32_t fk,
                                           int *st) {
    (void)fk;
    (void)st;
    const int hi = lane >> 4;
    const uint32_t lo16 = 16u * (lane & 15);
#pragma unroll
    for (int i = 0; i < 4; ++i) {  // head rows 2i, 2i + 1
        const int j = 2 * i + hi;
        if (j < H) {
            const uint32_t x = SLOS_IDX((uint32_t)(w.c + (hi ? w.hoff[2 * i + 1] : w.hoff[2 * i])), fk, st);
            cp_async16(stage + j * 256 + lo16, srcg + ((size_t)x << 8) + lo16);
        }
    }
    const uint32_t lc = (uint32_t)w.d.z;
#pragma unroll
    for (int i = 0; i < 4; ++i) {  // tail rows 8 + 2i, 9 + 2i
        const int q = 2 * i + hi;
        if (q < mL) {
            const uint32_t wd = i == 0 ? cr.x : (i == 1 ? cr.y : (i == 2 ? cr.z : cr.w));
            const uint32_t x = SLOS_IDX(lc + (hi ? (wd >> 16) : (wd & 0xffffu)), fk, st);
            cp_async16(stage + (8 + q) * 256 + lo16, srcg + ((size_t)x << 8) + lo16);
        }
    }
    if (!hi) cp_async16(stage + 16 * 256 + lo16, aprevg + ((size_t)w.c << 8) + lo16);
    if (SEED == SEED_BCAST) {
        int x = -1;
        if (lane < H) x = w.c + w.hl;
        else if (lane >= 8 && lane < 8 + mL) x = (int)(lc + crow16_rt(cr, lane - 8));
        if (x >= 0) cp_async4(stage + 17 * 256 + 4u * lane, seedb + x);
    }
}

template <int H, int SEED>
__global__ void __launch_bounds__(kSplitBwdWarps * 32, kSplitBwdMinBlocks) slos_bwd_ring_kernel(SplitBwdArgs a) {
    static_assert(SEED == SEED_G || SEED == SEED_BCAST || SEED == SEED_AMPS_T, "row seeds");
    __shared__ float2 red[kSplitBwdWarps][32];
    __shared__ uint32_t tmem_slot;
    extern __shared__ float4 ring_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int grp = blockIdx.y;
    const int inst = grp * kLanes + lane;
    const bool valid = inst < a.B;
    const int m = a.m;
    const int mL = m - H;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         static_cast<uint32_t>(__cvta_generic_to_shared(&tmem_slot))),
                     "r"(kSplitTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tq = tmem_slot + ((uint32_t)(warp * 32) << 16);
    {
        float z[16], uh[16], ut[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) z[i] = 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float2 u = make_float2(0.f, 0.f), v = make_float2(0.f, 0.f);
            if (valid && j < H) u = a.U[((int64_t)inst * m + j) * m + a.col];
            if (valid && j < mL) v = a.U[((int64_t)inst * m + H + j) * m + a.col];
            uh[2 * j] = u.x;
            uh[2 * j + 1] = u.y;
            ut[2 * j] = v.x;
            ut[2 * j + 1] = v.y;
        }
        tm_st16(tq, z);
        tm_st16(tq + 16, z);
        tm_st16(tq + 32, uh);
        tm_st16(tq + 48, ut);
    }
    // the warp's stages; the rows and seed slots no copy ever fills (modes past
    // the plan's) stay zero
    char *wring = reinterpret_cast<char *>(ring_raw) + (size_t)warp * kRingWarpBytes;
    const uint32_t wring_s = static_cast<uint32_t>(__cvta_generic_to_shared(wring));
#pragma unroll
    for (int s = 0; s < kRingDepth; ++s) {
        float2 *st = reinterpret_cast<float2 *>(wring + s * kRingStage);
        for (int j = H; j < 8; ++j) st[j * kLanes + lane] = make_float2(0.f, 0.f);
        for (int q = mL; q < 8; ++q) st[(8 + q) * kLanes + lane] = make_float2(0.f, 0.f);
        if (lane < 16) reinterpret_cast<float *>(st + 17 * kLanes)[lane] = 0.f;
    }
    __syncwarp();
    const size_t gprev = (size_t)grp * (size_t)a.Fprev * kLanes + lane;
    float2 *Gprevb = a.Gprev + gprev;
    // group bases (bytes): rows of 32 instances, 256 bytes each
    const size_t gk0 = (size_t)grp * (size_t)a.Fk * kLanes;
    const char *srcg = reinterpret_cast<const char *>(
        (SEED == SEED_G) ? a.Gk + gk0
                         : (SEED == SEED_AMPS_T) ? reinterpret_cast<const float2 *>(a.seed) + gk0 : a.an + gk0);
    const char *aprevg = reinterpret_cast<const char *>(a.aprev + (size_t)grp * (size_t)a.Fprev * kLanes);
    const float *seedb = reinterpret_cast<const float *>(a.seed);
    const int stride = gridDim.x * kSplitBwdWarps;
    const uint32_t fk = (uint32_t)a.Fk;
    int *const st = a.status;

    RingCursor cur;
    cur.ch = blockIdx.x * kSplitBwdWarps + warp;
    bool more = ring_run(cur, a, lane);
    uint4 cr = more ? __ldg(cur.crow) : make_uint4(0, 0, 0, 0);
    int cq[kRingDepth];  // parent of each stage in flight, oldest first
    int inflight = 0;
#pragma unroll
    for (int s = 0; s < kRingDepth; ++s) {
        cq[s] = -1;
        if (more) {
            ring_issue<H, SEED>(cur, cr, wring_s + s * kRingStage, lane, mL, srcg, aprevg, seedb, fk, st);
            cq[s] = cur.c;
            ++inflight;
            more = ring_next(cur, a, stride, lane);
            if (more) cr = __ldg(cur.crow);
        }
        cp_commit();
    }
    int s = 0;
    while (inflight > 0) {
        cp_wait<kRingDepth - 1>();
        __syncwarp();  // rows and seeds were copied by other lanes
        const float2 *stg = reinterpret_cast<const float2 *>(wring + s * kRingStage) + lane;
        const float2 av = stg[16 * kLanes];
        float2 gacc = make_float2(0.f, 0.f);
        const float4 *sd = reinterpret_cast<const float4 *>(wring + s * kRingStage + 17 * 256);
        // four tensor-memory batches (head modes 0..3, 4..H-1, tail modes 0..3, 4..7),
        // each reading its 4 children from the stage
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float2 g[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) g[i] = stg[(4 * q + i) * kLanes];
            if (SEED == SEED_BCAST) {
                const float4 v = sd[q];
                g[0] = cscale(g[0], v.x);
                g[1] = cscale(g[1], v.y);
                g[2] = cscale(g[2], v.z);
                g[3] = cscale(g[3], v.w);
            }
            if (q == 1)
                split_bwd_batch<H - 4>(tq, 8, 40, g, av, gacc);
            else
                split_bwd_batch<4>(tq, 8 * q, 32 + 8 * q, g, av, gacc);
        }
        Gprevb[(uint32_t)cq[0] << 5] = gacc;
        --inflight;
        __syncwarp();  // every lane has read this stage
        // refill the stage just read with the parent kRingDepth ahead
        const int cnew = more ? cur.c : -1;
        if (more) {
            ring_issue<H, SEED>(cur, cr, wring_s + s * kRingStage, lane, mL, srcg, aprevg, seedb, fk, st);
            ++inflight;
            more = ring_next(cur, a, stride, lane);
            if (more) cr = __ldg(cur.crow);
        }
        cp_commit();
#pragma unroll
        for (int i = 0; i + 1 < kRingDepth; ++i) cq[i] = cq[i + 1];
        cq[kRingDepth - 1] = cnew;
        s = (s + 1 == kRingDepth) ? 0 : s + 1;
    }
    cp_wait<0>();
    // reduce dU over the CTA's warps, one mode at a time
    float2 *dst = a.dUpart + (((int64_t)grp * gridDim.x + blockIdx.x) * kLanes) * m;
    {
        float dh[16], dt[16];
        tm_ld16(tq, dh);
        tm_ld16(tq + 16, dt);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (j < m) {
                red[warp][lane] = j < H ? make_float2(dh[2 * j], dh[2 * j + 1])
                                        : make_float2(dt[2 * (j - H)], dt[2 * (j - H) + 1]);
                __syncthreads();
                if (warp == 0) {
                    float2 t = red[0][lane];
#pragma unroll
                    for (int w = 1; w < kSplitBwdWarps; ++w) {
                        t.x += red[w][lane].x;
                        t.y += red[w][lane].y;
                    }
                    dst[lane * m + j] = t;
                }
                __syncthreads();
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_slot), "r"(kSplitTmemCols)
                     : "memory");
    }
}

// ============================================================ launchers
template <int H>
static cudaError_t launch_bwd_split_h(const SplitBwdArgs &a, int NG, int seed, int blocks_x, cudaStream_t s,
                                      bool fuse) {
    const int th = kSplitBwdWarps * 32;
    const dim3 grid(blocks_x, NG);
    const size_t rs = split_ring_smem_bytes();
    if (fuse) {
        if (seed != SEED_G) return cudaErrorInvalidValue;
        slos_bwd_split_kernel<H, SEED_G, true><<<grid, th, 0, s>>>(a);
        return cudaGetLastError();
    }
    switch (seed) {
        case SEED_G: slos_bwd_split_kernel<H, SEED_G><<<grid, th, 0, s>>>(a); break;
        case SEED_BCAST: slos_bwd_ring_kernel<H, SEED_BCAST><<<grid, th, rs, s>>>(a); break;
        case SEED_T: slos_bwd_split_kernel<H, SEED_T><<<grid, th, 0, s>>>(a); break;
        case SEED_AMPS_T: slos_bwd_ring_kernel<H, SEED_AMPS_T><<<grid, th, rs, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t slos_launch_bwd_split(const SplitBwdArgs &a, int NG, int seed, int h, int blocks_x, cudaStream_t s,
                                  bool fuse_prev) {
    switch (h) {
        case 6: return launch_bwd_split_h<6>(a, NG, seed, blocks_x, s, fuse_prev);
        case 8: return launch_bwd_split_h<8>(a, NG, seed, blocks_x, s, fuse_prev);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace slos
