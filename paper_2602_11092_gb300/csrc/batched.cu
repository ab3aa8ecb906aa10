// Uneven batches: instances of different (m, n, input, detection) in ONE
// persistent kernel launch (graph-capturable), with launch shapes picked by
// an autotuner.
//
// Instances with the same shape are packed 32 per "lane group" (lane =
// instance, as in the single-shape path).  Work item = (lane group, layer k,
// chunk of consecutive Fock states of layer k).  Items are listed layer by
// layer (all layer-1 items of every lane group, then all layer-2 items, ...),
// largest lane groups first inside a layer (longest-processing-time order).
// Warps pop items in that order with one atomic counter; an item of layer
// k >= 2 waits until every item of its lane group's layer k-1 has finished
// (a per-descriptor completion counter).  Every item an item waits on was
// popped earlier by a warp that is running, so the wait always ends; it is
// bounded anyway, and a wait that runs out records SLOS_ERR_TIMEOUT and the
// item id in the plan's status word and stops the warp.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/slos.h"
#include "common.cuh"
#include "plan.h"
#include "profile.h"

namespace slos {
slos_status_t fail(slos_status_t st, const std::string &msg);

constexpr int kBMax = 20;  // modes handled by the persistent kernel (m <= 20)

struct BShape {
    int m, n, det, K;
    int cols[kMaxPhotons];
    int64_t F[kMaxPhotons + 1];
    float inv_sfact;
    int pat_off[kMaxPhotons + 2];
};

struct BLaneGroup {
    int shape;
    int inst[kLanes];     // global instance index per lane, -1 = empty lane
    int64_t buf[2];       // workspace byte offsets of the two layer buffers
};

struct BDesc {
    int lg;      // lane group
    int k;       // layer
    int dep;     // descriptor of layer k-1 of the same lane group (-1 for k = 1)
    int nchunks;
};

struct BArgs {
    const BShape *shapes;
    const BLaneGroup *lgs;
    const BDesc *desc;
    const int64_t *first_item;  // [ndesc + 1]
    int ndesc;
    int64_t total_items;
    int chunk;
    const float2 *U;
    const int64_t *u_off;
    float *out;
    const int64_t *out_off;
    char *ws;
    int *done;          // [ndesc] completion counters (zeroed per launch)
    unsigned long long *head;  // work counter (zeroed per launch)
    int *status;        // plan status word
    long long spin_limit;
};

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <int MMAX>
__global__ void __launch_bounds__(256) slos_batched_kernel(BArgs a) {
    extern __shared__ float smem_b[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float *tile = smem_b + warp * (32 * 33);
    for (;;) {
        unsigned long long q = 0;
        if (lane == 0) q = atomicAdd(a.head, 1ull);
        q = __shfl_sync(0xffffffffu, q, 0);
        if ((int64_t)q >= a.total_items) break;
        // descriptor of item q: last i with first_item[i] <= q
        int lo = 0, hi = a.ndesc - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.first_item[mid] <= (int64_t)q) lo = mid;
            else hi = mid - 1;
        }
        const BDesc d = a.desc[lo];
        const int64_t chunk_id = (int64_t)q - a.first_item[lo];
        const BLaneGroup &g = a.lgs[d.lg];
        const BShape &sh = a.shapes[g.shape];
        const int m = sh.m, n = sh.n, k = d.k;
        if (d.dep >= 0) {
            const int need = a.desc[d.dep].nchunks;
            long long spins = 0;
            bool ok = true;
            if (lane == 0) {
                while (ld_acquire(a.done + d.dep) < need) {
                    if (++spins > a.spin_limit) {
                        ok = false;
                        break;
                    }
                    __nanosleep(200);
                }
                if (!ok) {
                    atomicCAS(a.status, 0, (int)SLOS_ERR_TIMEOUT);
                    atomicExch(a.status + 1, (int)q);
                }
            }
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) return;
            __threadfence();
        }
        const int inst = g.inst[lane];
        const bool valid = inst >= 0;
        const int col = sh.cols[k - 1];
        float2 u[MMAX];
#pragma unroll
        for (int j = 0; j < MMAX; ++j) {
            u[j] = make_float2(0.f, 0.f);
            if (j < m && valid) u[j] = a.U[a.u_off[inst] + (int64_t)j * m + col];
        }
        const int64_t Fk = sh.F[k], Fp = sh.F[k - 1];
        const float2 *prev = reinterpret_cast<const float2 *>(a.ws + g.buf[(n - 1 - (k - 1)) & 1]) + lane;
        float2 *next = reinterpret_cast<float2 *>(a.ws + g.buf[(n - 1 - k) & 1]) + lane;
        (void)Fp;
        const int L = k + m - 1;
        const int64_t c0 = chunk_id * a.chunk;
        const int64_t c1 = min(c0 + (int64_t)a.chunk, Fk);
        const bool final_layer = k == n;
        float *outp = (final_layer && valid) ? a.out + a.out_off[inst] : nullptr;
        int p[MMAX];
        unrank_bars<MMAX>(c0, m, L, p);
        int run_pat = -1;
        float run_val = 0.f;
        for (int64_t cs = c0; cs < c1; cs += 32) {
            const int64_t ce = min(cs + 32, c1);
            for (int64_t c = cs; c < ce; ++c) {
                float2 acc = make_float2(0.f, 0.f);
                int64_t S = 0;
                float fprod = 1.f;
                uint32_t supp = 0;
#pragma unroll
                for (int j = 0; j < MMAX; ++j) {
                    if (j < m) {
                        const int tj = occupation<MMAX>(j, m, L, p);
                        if (tj > 0) {
                            const float2 v = (k == 1) ? make_float2(1.f, 0.f) : __ldcg(prev + (c - S) * kLanes);
                            acc = cfma(u[j], v, acc);
                            fprod *= c_fact.v[tj];
                            supp |= 1u << j;
                        }
                        if (j < m - 1) S += (int64_t)binom_m1(p[j], m - 2 - j);
                    }
                }
                if (!final_layer) {
                    next[c * kLanes] = acc;
                } else {
                    const float pr = fprod * sh.inv_sfact * (acc.x * acc.x + acc.y * acc.y);
                    if (sh.det == SLOS_DETECT_THRESHOLD) {
                        const int pat = sh.pat_off[__popc(supp)] + (int)colex_rank(supp);
                        if (pat != run_pat) {
                            if (run_pat >= 0 && valid) atomicAdd(outp + run_pat, run_val);
                            run_pat = pat;
                            run_val = 0.f;
                        }
                        run_val += pr;
                    } else {
                        tile[lane * 33 + (int)(c - cs)] = pr;
                    }
                }
                next_bars<MMAX>(m, L, p);
            }
            if (final_layer && sh.det == SLOS_DETECT_PNR) {
                __syncwarp();
                const int nc = (int)(ce - cs);
                for (int i = 0; i < kLanes; ++i) {
                    const int ii = g.inst[i];
                    if (ii >= 0 && lane < nc) a.out[a.out_off[ii] + cs + lane] = tile[i * 33 + lane];
                }
                __syncwarp();
            }
        }
        if (final_layer && sh.det == SLOS_DETECT_THRESHOLD && run_pat >= 0 && valid) atomicAdd(outp + run_pat, run_val);
        __threadfence();
        __syncwarp();
        if (lane == 0) atomicAdd(a.done + lo, 1);
    }
}

struct BatchedPlan {
    int count = 0;
    std::vector<int> m, n, det;
    std::vector<std::vector<int>> s;
    std::vector<int64_t> u_off, out_off;
    std::vector<BShape> shapes;
    std::vector<BLaneGroup> lgs;
    std::string signature;
    // launch configuration (autotuned)
    int chunk = 128, threads = 256, blocks_per_sm = 2;
    // device copies (owned)
    BShape *d_shapes = nullptr;
    BLaneGroup *d_lgs = nullptr;
    BDesc *d_desc = nullptr;
    int64_t *d_first = nullptr, *d_uoff = nullptr, *d_ooff = nullptr;
    int ndesc = 0;
    int64_t total_items = 0;
    int built_chunk = -1;
    size_t layer_bytes = 0;  // workspace: layer buffers
    size_t ctrl_bytes = 0;   // workspace: counters
    int stall_desc = -1;     // a descriptor that others wait on (fault injection)
    bool inject_stall = false;
};

void batched_destroy(slos_plan_s *p) {
    BatchedPlan *b = p->batched;
    if (!b) return;
    cudaFree(b->d_shapes);
    cudaFree(b->d_lgs);
    cudaFree(b->d_desc);
    cudaFree(b->d_first);
    cudaFree(b->d_uoff);
    cudaFree(b->d_ooff);
    delete b;
    p->batched = nullptr;
}

// Descriptors and item offsets for a given chunk size (host build + upload).
static slos_status_t build_items(BatchedPlan *b, int chunk) {
    if (b->built_chunk == chunk) return SLOS_OK;
    struct D {
        BDesc d;
        int64_t work;
    };
    int kmax = 0;
    for (auto &sh : b->shapes) kmax = std::max(kmax, sh.n);
    std::vector<BDesc> desc;
    std::vector<int> idx_of((size_t)b->lgs.size() * (kmax + 1), -1);
    for (int k = 1; k <= kmax; ++k) {
        std::vector<D> layer;
        for (size_t l = 0; l < b->lgs.size(); ++l) {
            const BShape &sh = b->shapes[b->lgs[l].shape];
            if (k > sh.n) continue;
            D x;
            x.d.lg = (int)l;
            x.d.k = k;
            x.d.dep = -1;
            x.d.nchunks = (int)((sh.F[k] + chunk - 1) / chunk);
            x.work = sh.F[k] * sh.m;
            layer.push_back(x);
        }
        std::stable_sort(layer.begin(), layer.end(), [](const D &a, const D &c) { return a.work > c.work; });
        for (auto &x : layer) {
            x.d.dep = k > 1 ? idx_of[(size_t)x.d.lg * (kmax + 1) + k - 1] : -1;
            idx_of[(size_t)x.d.lg * (kmax + 1) + k] = (int)desc.size();
            desc.push_back(x.d);
        }
    }
    std::vector<int64_t> first(desc.size() + 1, 0);
    for (size_t i = 0; i < desc.size(); ++i) first[i + 1] = first[i] + desc[i].nchunks;
    cudaFree(b->d_desc);
    cudaFree(b->d_first);
    b->d_desc = nullptr;
    b->d_first = nullptr;
    if (cudaMalloc(&b->d_desc, std::max<size_t>(1, desc.size()) * sizeof(BDesc)) != cudaSuccess ||
        cudaMalloc(&b->d_first, first.size() * sizeof(int64_t)) != cudaSuccess)
        return fail(SLOS_ERR_OOM, "slos_batched_plan: cannot allocate work descriptors");
    cudaMemcpy(b->d_desc, desc.data(), desc.size() * sizeof(BDesc), cudaMemcpyHostToDevice);
    cudaMemcpy(b->d_first, first.data(), first.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    b->ndesc = (int)desc.size();
    b->total_items = first.back();
    b->stall_desc = -1;
    for (auto &d : desc)
        if (d.dep >= 0) {
            b->stall_desc = d.dep;
            break;
        }
    b->built_chunk = chunk;
    b->ctrl_bytes = align_up(sizeof(unsigned long long)) + align_up((size_t)b->ndesc * sizeof(int));
    return SLOS_OK;
}

static slos_status_t batched_launch(slos_plan_s *p, const void *U, float *out, void *ws, size_t ws_bytes,
                                    cudaStream_t s, int chunk, int threads, int bps) {
    BatchedPlan *b = p->batched;
    slos_status_t st = build_items(b, chunk);
    if (st != SLOS_OK) return st;
    const size_t need = b->layer_bytes + b->ctrl_bytes;
    if (ws_bytes < need || !ws) return fail(SLOS_ERR_INVALID_ARG, "slos_batched_forward: workspace too small");
    char *w = reinterpret_cast<char *>(ws);
    unsigned long long *head = reinterpret_cast<unsigned long long *>(w + b->layer_bytes);
    int *done = reinterpret_cast<int *>(w + b->layer_bytes + align_up(sizeof(unsigned long long)));
    cudaError_t e;
    if ((e = cudaMemsetAsync(w + b->layer_bytes, 0, b->ctrl_bytes, s)) != cudaSuccess)
        return fail(SLOS_ERR_CUDA, std::string("slos_batched_forward: ") + cudaGetErrorString(e));
    // threshold outputs accumulate: clear the packed output
    if ((e = cudaMemsetAsync(out, 0, (size_t)b->out_off[b->count] * sizeof(float), s)) != cudaSuccess)
        return fail(SLOS_ERR_CUDA, std::string("slos_batched_forward: ") + cudaGetErrorString(e));
    BArgs a;
    a.shapes = b->d_shapes;
    a.lgs = b->d_lgs;
    a.desc = b->d_desc;
    a.first_item = b->d_first;
    a.ndesc = b->ndesc;
    a.total_items = b->total_items;
    a.chunk = chunk;
    a.U = reinterpret_cast<const float2 *>(U);
    a.u_off = b->d_uoff;
    a.out = out;
    a.out_off = b->d_ooff;
    a.ws = w;
    a.done = done;
    a.head = head;
    a.status = p->d_status;
    a.spin_limit = 20000000;  // ~4 s of 200 ns sleeps: far beyond any layer
    if (b->inject_stall && b->stall_desc >= 0) {
        // fault injection: this completion counter starts hugely negative, so
        // the items waiting on it never see it complete; short wait limit
        if ((e = cudaMemsetAsync(done + b->stall_desc, 0x80, sizeof(int), s)) != cudaSuccess)
            return fail(SLOS_ERR_CUDA, std::string("slos_batched_forward: ") + cudaGetErrorString(e));
        a.spin_limit = 5000;
    }
    const int warps = threads / 32;
    const size_t smem = (size_t)warps * 32 * 33 * sizeof(float);
    const int grid = std::max(1, p->sm_count * bps);
    double bytes = 0.0;
    for (int i = 0; i < b->count; ++i) bytes += 4.0 * (b->out_off[i + 1] - b->out_off[i]);
    ProfScope ps("slos_batched", bytes, s);
    slos_batched_kernel<kBMax><<<grid, threads, smem, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return fail(SLOS_ERR_CUDA, std::string("slos_batched_forward: ") + cudaGetErrorString(e));
    return SLOS_OK;
}

// ---------------------------------------------------------------- autotune cache
static std::string device_name(int dev) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    return prop.name;
}

static bool cache_lookup(const std::string &path, const std::string &key, int *chunk, int *threads, int *bps) {
    std::ifstream f(path);
    if (!f) return false;
    std::string line;
    while (std::getline(f, line)) {
        // one JSON object per line: {"key": "...", "chunk": C, "threads": T, "blocks_per_sm": B, "ms": X}
        const std::string kq = "\"key\": \"" + key + "\"";
        if (line.find(kq) == std::string::npos) continue;
        auto num = [&](const char *name, int *dst) {
            const std::string nq = std::string("\"") + name + "\": ";
            size_t pos = line.find(nq);
            if (pos == std::string::npos) return false;
            *dst = atoi(line.c_str() + pos + nq.size());
            return true;
        };
        return num("chunk", chunk) && num("threads", threads) && num("blocks_per_sm", bps);
    }
    return false;
}

}  // namespace slos

using namespace slos;

extern "C" {

slos_status_t slos_batched_plan(int count, const int *m, const int *n, const int *const *input_states,
                                const slos_detection_t *detection, slos_plan_t *out) {
    if (!out) return fail(SLOS_ERR_INVALID_ARG, "slos_batched_plan: NULL out");
    *out = nullptr;
    if (count <= 0 || !m || !n || !input_states || !detection)
        return fail(SLOS_ERR_INVALID_ARG, "slos_batched_plan: bad arguments");
    BatchedPlan *b = new BatchedPlan();
    b->count = count;
    std::map<std::vector<int>, int> shape_of;  // (m, det, s...) -> shape index
    std::vector<std::vector<int>> members;
    std::vector<int> shape_idx(count);
    std::ostringstream sig;
    for (int i = 0; i < count; ++i) {
        const int mi = m[i], ni = n[i];
        if (mi < 2 || mi > kBMax || ni < 1 || ni > kMaxPhotons) {
            delete b;
            return fail(SLOS_ERR_UNSUPPORTED, "slos_batched_plan: instance " + std::to_string(i) +
                                                  " needs 2 <= m <= 20 and 1 <= n <= 12");
        }
        if (detection[i] != SLOS_DETECT_PNR && detection[i] != SLOS_DETECT_THRESHOLD) {
            delete b;
            return fail(SLOS_ERR_INVALID_ARG, "slos_batched_plan: unknown detection");
        }
        std::vector<int> key = {mi, (int)detection[i]};
        int tot = 0;
        for (int q = 0; q < mi; ++q) {
            if (input_states[i][q] < 0) {
                delete b;
                return fail(SLOS_ERR_INVALID_ARG, "slos_batched_plan: negative occupation");
            }
            tot += input_states[i][q];
            key.push_back(input_states[i][q]);
        }
        if (tot != ni) {
            delete b;
            return fail(SLOS_ERR_INVALID_ARG, "slos_batched_plan: input state of instance " + std::to_string(i) +
                                                  " does not hold n photons");
        }
        auto it = shape_of.find(key);
        int si;
        if (it == shape_of.end()) {
            si = (int)b->shapes.size();
            shape_of[key] = si;
            BShape sh;
            memset(&sh, 0, sizeof(sh));
            sh.m = mi;
            sh.n = ni;
            sh.det = (int)detection[i];
            int c = 0;
            double sf = 1.0;
            for (int q = 0; q < mi; ++q)
                for (int r = 0; r < input_states[i][q]; ++r) {
                    sh.cols[c++] = q;
                    if (r >= 1) sf *= (r + 1);
                }
            sh.inv_sfact = (float)(1.0 / sf);
            for (int k = 0; k <= ni; ++k) sh.F[k] = binom_host(mi + k - 1, k);
            int64_t acc = 0;
            for (int j = 1; j <= std::min(ni, mi); ++j) {
                sh.pat_off[j] = (int)acc;
                acc += binom_host(mi, j);
            }
            sh.K = (int)(detection[i] == SLOS_DETECT_PNR ? sh.F[ni] : acc);
            b->shapes.push_back(sh);
            members.emplace_back();
        } else {
            si = it->second;
        }
        members[si].push_back(i);
        shape_idx[i] = si;
        b->m.push_back(mi);
        b->n.push_back(ni);
        b->det.push_back((int)detection[i]);
        b->s.emplace_back(input_states[i], input_states[i] + mi);
        sig << mi << "," << ni << "," << (int)detection[i] << ";";
    }
    // packed offsets in instance order
    b->u_off.assign(count + 1, 0);
    b->out_off.assign(count + 1, 0);
    for (int i = 0; i < count; ++i) {
        b->u_off[i + 1] = b->u_off[i] + (int64_t)b->m[i] * b->m[i];
        b->out_off[i + 1] = b->out_off[i] + b->shapes[shape_idx[i]].K;
    }
    // lane groups and their layer buffers
    size_t off = 0;
    for (size_t si = 0; si < members.size(); ++si) {
        const BShape &sh = b->shapes[si];
        for (size_t q = 0; q < members[si].size(); q += kLanes) {
            BLaneGroup g;
            g.shape = (int)si;
            for (int l = 0; l < kLanes; ++l)
                g.inst[l] = q + l < members[si].size() ? members[si][q + l] : -1;
            const int64_t f1 = sh.n >= 2 ? sh.F[sh.n - 1] : 1;
            const int64_t f2 = sh.n >= 3 ? sh.F[sh.n - 2] : 1;
            g.buf[0] = (int64_t)off;
            off += align_up((size_t)f1 * kLanes * sizeof(float2));
            g.buf[1] = (int64_t)off;
            off += align_up((size_t)f2 * kLanes * sizeof(float2));
            b->lgs.push_back(g);
        }
    }
    b->layer_bytes = off;
    b->signature = sig.str();
    slos_plan_s *p = new slos_plan_s();
    p->kind = 1;
    p->m = 0;
    p->n = 0;
    p->batched = b;
    p->d_status = nullptr;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete b;
        delete p;
        return fail(SLOS_ERR_CUDA, "slos_batched_plan: no CUDA device");
    }
    cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device);
    if (p->sm_count <= 0) p->sm_count = 148;
    auto cleanup = [&](const char *msg) {
        batched_destroy(p);
        if (p->d_status) cudaFree(p->d_status);
        delete p;
        return fail(SLOS_ERR_OOM, msg);
    };
    if (cudaMalloc(&p->d_status, 64) != cudaSuccess) return cleanup("slos_batched_plan: status word");
    cudaMemset(p->d_status, 0, 64);
    if (cudaMalloc(&b->d_shapes, b->shapes.size() * sizeof(BShape)) != cudaSuccess ||
        cudaMalloc(&b->d_lgs, b->lgs.size() * sizeof(BLaneGroup)) != cudaSuccess ||
        cudaMalloc(&b->d_uoff, b->u_off.size() * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc(&b->d_ooff, b->out_off.size() * sizeof(int64_t)) != cudaSuccess)
        return cleanup("slos_batched_plan: descriptor tables");
    cudaMemcpy(b->d_shapes, b->shapes.data(), b->shapes.size() * sizeof(BShape), cudaMemcpyHostToDevice);
    cudaMemcpy(b->d_lgs, b->lgs.data(), b->lgs.size() * sizeof(BLaneGroup), cudaMemcpyHostToDevice);
    cudaMemcpy(b->d_uoff, b->u_off.data(), b->u_off.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    cudaMemcpy(b->d_ooff, b->out_off.data(), b->out_off.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    slos_status_t st = build_items(b, b->chunk);
    if (st != SLOS_OK) {
        batched_destroy(p);
        cudaFree(p->d_status);
        delete p;
        return st;
    }
    *out = p;
    return SLOS_OK;
}

slos_status_t slos_batched_query(slos_plan_t p, int64_t *u_offsets, int64_t *out_offsets, size_t *workspace_bytes) {
    if (!p || p->kind != 1 || !p->batched) return fail(SLOS_ERR_INVALID_ARG, "slos_batched_query: not a batched plan");
    BatchedPlan *b = p->batched;
    if (u_offsets) memcpy(u_offsets, b->u_off.data(), b->u_off.size() * sizeof(int64_t));
    if (out_offsets) memcpy(out_offsets, b->out_off.data(), b->out_off.size() * sizeof(int64_t));
    if (workspace_bytes) {
        // enough for the largest chunk the autotuner tries (smallest chunk = most descriptors is the same count)
        *workspace_bytes = b->layer_bytes + align_up(sizeof(unsigned long long)) +
                           align_up((size_t)b->lgs.size() * (kMaxPhotons + 1) * sizeof(int));
    }
    return SLOS_OK;
}

slos_status_t slos_batched_forward(slos_plan_t p, const void *U_packed, float *out_packed, void *workspace,
                                   size_t workspace_bytes, void *stream) {
    if (!p || p->kind != 1 || !p->batched) return fail(SLOS_ERR_INVALID_ARG, "slos_batched_forward: not a batched plan");
    if (!U_packed || !out_packed) return fail(SLOS_ERR_INVALID_ARG, "slos_batched_forward: NULL pointer");
    BatchedPlan *b = p->batched;
    return batched_launch(p, U_packed, out_packed, workspace, workspace_bytes, (cudaStream_t)stream, b->chunk,
                          b->threads, b->blocks_per_sm);
}

slos_status_t slos_batched_inject_stall(slos_plan_t p, int enable) {
    if (!p || p->kind != 1 || !p->batched) return fail(SLOS_ERR_INVALID_ARG, "slos_batched_inject_stall: not a batched plan");
    p->batched->inject_stall = enable != 0;
    return SLOS_OK;
}

slos_status_t slos_batched_autotune(slos_plan_t p, const void *U_packed, float *out_packed, void *workspace,
                                    size_t workspace_bytes, const char *cache_path, void *stream) {
    if (!p || p->kind != 1 || !p->batched) return fail(SLOS_ERR_INVALID_ARG, "slos_batched_autotune: not a batched plan");
    BatchedPlan *b = p->batched;
    cudaStream_t s = (cudaStream_t)stream;
    const std::string key = device_name(p->device) + "|" + std::to_string(std::hash<std::string>()(b->signature));
    int c = 0, t = 0, bp = 0;
    if (cache_path && cache_lookup(cache_path, key, &c, &t, &bp)) {
        b->chunk = c;
        b->threads = t;
        b->blocks_per_sm = bp;
        return build_items(b, c);
    }
    const int chunks[] = {64, 128, 256, 512};
    const int thread_opts[] = {128, 256};
    const int bps_opts[] = {1, 2, 3, 4};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int bc = b->chunk, bt = b->threads, bb = b->blocks_per_sm;
    for (int ch : chunks) {
        for (int th : thread_opts) {
            for (int bps : bps_opts) {
                int nb = 0;
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, slos_batched_kernel<kBMax>, th,
                                                              (size_t)(th / 32) * 32 * 33 * sizeof(float));
                if (nb < bps) continue;  // a persistent grid must be fully resident
                slos_status_t st = batched_launch(p, U_packed, out_packed, workspace, workspace_bytes, s, ch, th, bps);
                if (st != SLOS_OK) return st;  // warm-up (also builds the items)
                cudaEventRecord(e0, s);
                for (int r = 0; r < 2; ++r) {
                    st = batched_launch(p, U_packed, out_packed, workspace, workspace_bytes, s, ch, th, bps);
                    if (st != SLOS_OK) return st;
                }
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) return fail(SLOS_ERR_CUDA, "slos_batched_autotune: sync");
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                ms *= 0.5f;
                if (ms < best) {
                    best = ms;
                    bc = ch;
                    bt = th;
                    bb = bps;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->chunk = bc;
    b->threads = bt;
    b->blocks_per_sm = bb;
    if (cache_path) {
        std::ofstream f(cache_path, std::ios::app);
        if (f) {
            f << "{\"key\": \"" << key << "\", \"chunk\": " << bc << ", \"threads\": " << bt
              << ", \"blocks_per_sm\": " << bb << ", \"ms\": " << best << "}\n";
        }
    }
    return build_items(b, bc);
}

}  // extern "C"
