// Batched interferometer mesh -> unitary (forward) and its reverse sweep
// (backward).  Sec. II-A.3: the trainable parameters are the phases of the
// physical components; Sec. II-C.1: U(x, theta) = W2(theta2) S(x) W1(theta1).
//
// One warp per instance.  Lane i carries column i of the running product
// X = T_l ... T_1 in registers; an MZI on modes (k, k+1) only mixes entries
// k and k+1 of every column, so each lane updates its own column and no data
// moves between lanes.  The rectangular layout is regular (column c holds the
// pairs k = c mod 2, c mod 2 + 2, ...), so the pair index k is a compile-time
// constant inside the unrolled inner loop and the column stays in registers.
//
// MZI(theta, phi) = B diag(e^{i theta}, 1) B diag(e^{i phi}, 1),
// B = [[1, i], [i, 1]]/sqrt 2, which multiplies out to
//     i e^{i theta/2} [[sin(theta/2) e^{i phi},  cos(theta/2)],
//                      [cos(theta/2) e^{i phi}, -sin(theta/2)]].
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "common.cuh"
#include "mesh.h"
#include "profile.h"

namespace slos {

struct Mzi {
    float2 t00, t01, t10, t11;
    float2 eth, eph;  // e^{i theta}, e^{i phi}
};

__device__ __forceinline__ Mzi make_mzi(float theta, float phi) {
    float sh, chh, sp, cp, st, ct;
    sincosf(0.5f * theta, &sh, &chh);
    sincosf(phi, &sp, &cp);
    sincosf(theta, &st, &ct);
    // g = i e^{i theta/2} = (-sin(theta/2), cos(theta/2))
    const float2 g = make_float2(-sh, chh);
    const float2 eph = make_float2(cp, sp);
    Mzi z;
    z.t01 = cscale(g, chh);
    z.t11 = cscale(g, -sh);
    z.t00 = cmul(cscale(g, sh), eph);
    z.t10 = cmul(cscale(g, chh), eph);
    z.eth = make_float2(ct, st);
    z.eph = eph;
    return z;
}

__device__ __forceinline__ int mzi_offset(int c, int m) {
    const int ne = m / 2, no = (m - 1) / 2;  // MZIs in even / odd columns
    return ((c + 1) / 2) * ne + (c / 2) * no;
}

// The 2x2 blocks of every MZI (and the data-screen phase factors) of one
// instance, computed in parallel by the warp's lanes into shared memory, so
// the sequential sweeps below only read them.
struct MziTab {
    float2 t00, t01, t10, t11, eth, eph;
};

__device__ __forceinline__ void fill_mzi_table(const float *th, const float *dd, const float *dw, int m, int n_data,
                                               int lane, MziTab *tab, float2 *ed) {
    const int nmzi = m * (m - 1) / 2;
    for (int idx = lane; idx < nmzi; idx += 32) {
        const Mzi z = make_mzi(th[2 * idx], th[2 * idx + 1]);
        tab[idx] = MziTab{z.t00, z.t01, z.t10, z.t11, z.eth, z.eph};
    }
    for (int j = lane; j < n_data; j += 32) {
        float s, c;
        sincosf(dw ? dd[j] * dw[j] : dd[j], &s, &c);
        ed[j] = make_float2(c, s);
    }
    __syncwarp();
}

// Forward sweep for one column of U (lane = input mode), all in registers.
template <int MMAX>
__device__ __forceinline__ void mesh_column(const MziTab *tab, const float2 *ed, int m, int n_data, int data_col,
                                            int lane, float2 (&x)[MMAX]) {
#pragma unroll
    for (int j = 0; j < MMAX; ++j) x[j] = make_float2(j == lane ? 1.f : 0.f, 0.f);
    for (int c = 0; c <= m; ++c) {
        if (c == data_col && n_data > 0) {
#pragma unroll
            for (int j = 0; j < MMAX; ++j)
                if (j < n_data) x[j] = cmul(ed[j], x[j]);
        }
        if (c == m) break;
        const int base = mzi_offset(c, m);
        const int par = c & 1;
#pragma unroll
        for (int k = 0; k < MMAX - 1; ++k) {
            if ((k & 1) == par && k + 1 < m) {
                const MziTab z = tab[base + (k - par) / 2];
                const float2 xk = x[k], xk1 = x[k + 1];
                x[k] = cfma(z.t01, xk1, cmul(z.t00, xk));
                x[k + 1] = cfma(z.t11, xk1, cmul(z.t10, xk));
            }
        }
    }
}

// per-warp shared memory: MZI table + data-screen factors
template <int MMAX>
struct MeshSmem {
    MziTab tab[MMAX * (MMAX - 1) / 2];
    float2 ed[MMAX];
};

// warps (instances) per block of the forward mesh kernel: the per-warp MZI
// tables must stay under the 48 KB static shared-memory limit
template <int MMAX>
constexpr int mesh_fwd_warps() { return MMAX > 16 ? 2 : 4; }

template <int MMAX>
__global__ void mesh_fwd_kernel(MeshArgs a) {
    __shared__ MeshSmem<MMAX> sm[mesh_fwd_warps<MMAX>()];
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int b = blockIdx.x * (blockDim.x >> 5) + w;
    if (b >= a.B) return;
    const int m = a.m;
    const float *th = a.theta + (int64_t)b * a.theta_stride;
    const float *dd = a.data ? a.data + (int64_t)b * a.data_stride : nullptr;
    fill_mzi_table(th, dd, a.data_w, m, a.n_data, lane, sm[w].tab, sm[w].ed);
    float2 x[MMAX];
    mesh_column<MMAX>(sm[w].tab, sm[w].ed, m, a.n_data, a.data_col, lane, x);
    if (lane < m) {
        float2 *U = a.U + (int64_t)b * m * m;
#pragma unroll
        for (int j = 0; j < MMAX; ++j)
            if (j < m) U[j * m + lane] = x[j];
    }
}

// Reverse sweep.  With U = Y_l T_l X_{l-1} (X_{l-1} = T_{l-1}..T_1,
// Y_l = T_L..T_{l+1}) and M_l = Y_l^H dU, the gradient w.r.t. the 2x2 block
// is G = M_l X_{l-1}^H on rows/cols (k, k+1), and
//      dL/dx = Re sum_ab conj(G_ab) dT_ab/dx
//            = sum_i Re sum_ab conj(M_l[a][i]) X_{l-1}[b][i] dT_ab/dx,
// a sum over the columns i (lanes) of per-lane scalars.  Going down:
// X_{l-1} = T_l^H X_l, M_{l-1} = T_l^H M_l.  Each lane writes its scalar for
// every phase to shared memory during the sweep (no cross-lane traffic in
// the sequential part); the column sums are formed at the end, one phase per
// lane at a time, in a fixed order.
template <int MMAX>
__global__ void mesh_bwd_kernel(MeshBwdArgs a) {
    extern __shared__ float contrib[];  // [P + n_data][33]
    __shared__ MeshSmem<MMAX> sm;
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x;
    if (b >= a.B) return;
    const int m = a.m;
    const int P = m * (m - 1);
    const float *th = a.theta + (int64_t)b * a.theta_stride;
    const float *dd = a.data ? a.data + (int64_t)b * a.data_stride : nullptr;
    float *gth = a.dtheta + (int64_t)b * a.dtheta_stride;
    float2 x[MMAX], mm[MMAX];
    fill_mzi_table(th, dd, a.data_w, m, a.n_data, lane, sm.tab, sm.ed);
    mesh_column<MMAX>(sm.tab, sm.ed, m, a.n_data, a.data_col, lane, x);  // X = U, recomputed
#pragma unroll
    for (int j = 0; j < MMAX; ++j) {
        mm[j] = make_float2(0.f, 0.f);
        if (j < m && lane < m) mm[j] = a.dU[((int64_t)b * m + j) * m + lane];
        if (lane >= m) x[j] = make_float2(0.f, 0.f);
    }
    for (int c = m; c >= 0; --c) {
        if (c < m) {
            const int base = mzi_offset(c, m);
            const int par = c & 1;
#pragma unroll
            for (int k = 0; k < MMAX - 1; ++k) {
                if ((k & 1) == par && k + 1 < m) {
                    const int idx = base + (k - par) / 2;
                    const MziTab z = sm.tab[idx];  // precomputed by fill_mzi_table
                    // X_before = T^H X
                    const float2 xk = x[k], xk1 = x[k + 1];
                    const float2 bk = cfma_conj_a(z.t10, xk1, make_float2(z.t00.x * xk.x + z.t00.y * xk.y,
                                                                           z.t00.x * xk.y - z.t00.y * xk.x));
                    const float2 bk1 = cfma_conj_a(z.t11, xk1, make_float2(z.t01.x * xk.x + z.t01.y * xk.y,
                                                                            z.t01.x * xk.y - z.t01.y * xk.x));
                    x[k] = bk;
                    x[k + 1] = bk1;
                    const float2 mk = mm[k], mk1 = mm[k + 1];
                    // dT/dtheta = [[ (i/2) e^{i th} e^{i ph}, -(1/2) e^{i th}],
                    //              [-(1/2) e^{i th} e^{i ph}, -(i/2) e^{i th}]]
                    const float2 e2 = cmul(z.eth, z.eph);
                    const float2 d00 = make_float2(-0.5f * e2.y, 0.5f * e2.x);
                    const float2 d01 = make_float2(-0.5f * z.eth.x, -0.5f * z.eth.y);
                    const float2 d10 = make_float2(-0.5f * e2.x, -0.5f * e2.y);
                    const float2 d11 = make_float2(0.5f * z.eth.y, -0.5f * z.eth.x);
                    // dT/dphi = [[i t00, 0], [i t10, 0]]
                    const float2 p00 = make_float2(-z.t00.y, z.t00.x);
                    const float2 p10 = make_float2(-z.t10.y, z.t10.x);
                    // per-lane Re( conj(M_a) sum_b Xb_b dT_ab )
                    const float2 r0 = cfma(bk1, d01, cmul(bk, d00));
                    const float2 r1 = cfma(bk1, d11, cmul(bk, d10));
                    const float cth = mk.x * r0.x + mk.y * r0.y + mk1.x * r1.x + mk1.y * r1.y;
                    const float2 q0 = cmul(bk, p00), q1 = cmul(bk, p10);
                    const float cph = mk.x * q0.x + mk.y * q0.y + mk1.x * q1.x + mk1.y * q1.y;
                    contrib[(2 * idx) * 33 + lane] = cth;
                    contrib[(2 * idx + 1) * 33 + lane] = cph;
                    // M_before = T^H M
                    mm[k] = cfma_conj_a(z.t10, mk1, make_float2(z.t00.x * mk.x + z.t00.y * mk.y,
                                                                z.t00.x * mk.y - z.t00.y * mk.x));
                    mm[k + 1] = cfma_conj_a(z.t11, mk1, make_float2(z.t01.x * mk.x + z.t01.y * mk.y,
                                                                    z.t01.x * mk.y - z.t01.y * mk.x));
                }
            }
        }
        if (c == a.data_col && a.n_data > 0) {
#pragma unroll
            for (int j = 0; j < MMAX; ++j) {
                if (j < a.n_data) {
                    const float2 e = sm.ed[j];
                    // X_before = conj(e) X ; contribution Re(conj(M) Xb (i e))
                    const float2 xb = make_float2(e.x * x[j].x + e.y * x[j].y, e.x * x[j].y - e.y * x[j].x);
                    x[j] = xb;
                    const float2 r = cmul(xb, make_float2(-e.y, e.x));
                    contrib[(P + j) * 33 + lane] = mm[j].x * r.x + mm[j].y * r.y;
                    mm[j] = make_float2(e.x * mm[j].x + e.y * mm[j].y, e.x * mm[j].y - e.y * mm[j].x);
                }
            }
        }
    }
    __syncwarp();
    for (int q = lane; q < P + a.n_data; q += 32) {
        float sum = 0.f;
        for (int l = 0; l < 32; ++l) sum += contrib[q * 33 + l];
        if (q < P) gth[q] = sum;
        else {
            // d/dx_j = d/dphi_j * w_j, d/dw_j = d/dphi_j * x_j (phi_j = x_j w_j)
            const int j = q - P;
            a.ddata[(int64_t)b * a.n_data + j] = a.data_w ? sum * a.data_w[j] : sum;
            if (a.dw) a.dw[(int64_t)b * a.n_data + j] = sum * dd[j];
        }
    }
}

// out[p] = sum_b part[b][p] for rows b < B of P floats, in a fixed order: a
// block takes 32 consecutive columns; warp w sums rows w, w + 8, w + 16, ...
// in row order (coalesced 128-byte row pieces, several loads in flight), and
// the 8 partial sums are added in warp order.
constexpr int kReduceWarps = 8;
__global__ void __launch_bounds__(kReduceWarps * 32) mesh_reduce_kernel(const float *part, int B, int P, float *out) {
    __shared__ float red[kReduceWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int p = blockIdx.x * 32 + lane;
    float s = 0.f;
    if (p < P) {
#pragma unroll 4
        for (int b = warp; b < B; b += kReduceWarps) s += part[(int64_t)b * P + p];
    }
    red[warp][lane] = s;
    __syncthreads();
    if (warp == 0 && p < P) {
        float t = red[0][lane];
#pragma unroll
        for (int w = 1; w < kReduceWarps; ++w) t += red[w][lane];
        out[p] = t;
    }
}

cudaError_t mesh_sum_rows_launch(const float *part, int B, int P, float *out, cudaStream_t s) {
    count_launch();
    mesh_reduce_kernel<<<(P + 31) / 32, kReduceWarps * 32, 0, s>>>(part, B, P, out);
    return cudaGetLastError();
}

template <int MMAX>
static cudaError_t launch_fwd(const MeshArgs &a, cudaStream_t s) {
    const int wpb = mesh_fwd_warps<MMAX>();
    mesh_fwd_kernel<MMAX><<<(a.B + wpb - 1) / wpb, wpb * 32, 0, s>>>(a);
    return cudaGetLastError();
}

template <int MMAX>
static cudaError_t launch_bwd(const MeshBwdArgs &a, cudaStream_t s) {
    const size_t smem = (size_t)(a.m * (a.m - 1) + a.n_data) * 33 * sizeof(float);
    // the attribute belongs to the current device's context: set it once per device
    // (largest case: m = 24 needs 76 KB)
    static std::mutex mu;
    static bool attr_set[64] = {false};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!attr_set[dev]) {
            cudaError_t e = cudaFuncSetAttribute(mesh_bwd_kernel<MMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)((24 * 23 + 24) * 33 * sizeof(float)));
            if (e != cudaSuccess) return e;
            attr_set[dev] = true;
        }
    }
    mesh_bwd_kernel<MMAX><<<a.B, 32, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t mesh_forward_launch(const MeshArgs &a, cudaStream_t s) {
    if (a.B == 0) return cudaSuccess;
    if (a.m <= 8) return launch_fwd<8>(a, s);
    if (a.m <= 16) return launch_fwd<16>(a, s);
    return launch_fwd<24>(a, s);
}

cudaError_t mesh_backward_launch(const MeshBwdArgs &a, float *dtheta_shared, cudaStream_t s) {
    if (a.B == 0) return cudaSuccess;
    cudaError_t e;
    if (a.m <= 8) e = launch_bwd<8>(a, s);
    else if (a.m <= 16) e = launch_bwd<16>(a, s);
    else e = launch_bwd<24>(a, s);
    if (e != cudaSuccess) return e;
    if (dtheta_shared) {
        const int P = a.m * (a.m - 1);
        e = mesh_sum_rows_launch(a.dtheta, a.B, P, dtheta_shared, s);
    }
    return e;
}

}  // namespace slos
