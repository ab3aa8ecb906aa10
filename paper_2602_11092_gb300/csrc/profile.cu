// Launch counting and optional per-launch CUDA-event timing.
#include <cuda_runtime.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/slos.h"
#include "profile.h"

namespace slos {
slos_status_t fail(slos_status_t st, const std::string &msg);

namespace {
struct Rec {
    std::string name;
    cudaEvent_t a, b;
    double bytes;
};
struct Agg {
    std::string name;
    int64_t launches;
    double ms, bytes;
};
std::atomic<int64_t> g_launches{0};
std::atomic<bool> g_enabled{false};
std::mutex g_mu;
std::vector<Rec> g_recs;
std::vector<Rec> g_pool;  // reusable event pairs
std::vector<Agg> g_aggs;
}  // namespace

// Every launch is also an NVTX range named after it (a no-op unless a
// profiler that collects NVTX is attached).
ProfScope::ProfScope(const char *name, double bytes, cudaStream_t s) : active_(false), stream_(s) {
    nvtxRangePushA(name);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_enabled.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lk(g_mu);
    Rec r;
    if (!g_pool.empty()) {
        r = g_pool.back();
        g_pool.pop_back();
    } else {
        if (cudaEventCreate(&r.a) != cudaSuccess) return;
        if (cudaEventCreate(&r.b) != cudaSuccess) {
            cudaEventDestroy(r.a);
            return;
        }
    }
    r.name = name;
    r.bytes = bytes;
    cudaEventRecord(r.a, s);
    g_recs.push_back(r);
    idx_ = g_recs.size() - 1;
    active_ = true;
}

ProfScope::~ProfScope() {
    nvtxRangePop();
    if (!active_) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (idx_ < g_recs.size()) cudaEventRecord(g_recs[idx_].b, stream_);
}

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

}  // namespace slos

using namespace slos;

extern "C" {

slos_status_t slos_profile_enable(int enable) {
    g_enabled.store(enable != 0);
    return SLOS_OK;
}

slos_status_t slos_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &r : g_recs) g_pool.push_back(r);
    g_recs.clear();
    g_aggs.clear();
    g_launches.store(0);
    return SLOS_OK;
}

int64_t slos_launch_count(void) { return g_launches.load(); }

int slos_profile_collect(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    std::map<std::string, size_t> pos;
    g_aggs.clear();
    for (auto &r : g_recs) {
        if (cudaEventSynchronize(r.b) != cudaSuccess) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) continue;
        auto it = pos.find(r.name);
        if (it == pos.end()) {
            pos[r.name] = g_aggs.size();
            g_aggs.push_back(Agg{r.name, 1, (double)ms, r.bytes});
        } else {
            Agg &a = g_aggs[it->second];
            a.launches += 1;
            a.ms += ms;
            a.bytes += r.bytes;
        }
    }
    return (int)g_aggs.size();
}

slos_status_t slos_profile_entry(int i, char *name, size_t name_len, int64_t *launches, double *total_ms,
                                 double *total_bytes) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (i < 0 || i >= (int)g_aggs.size()) return fail(SLOS_ERR_INVALID_ARG, "slos_profile_entry: index");
    const Agg &a = g_aggs[i];
    if (name && name_len > 0) {
        strncpy(name, a.name.c_str(), name_len - 1);
        name[name_len - 1] = 0;
    }
    if (launches) *launches = a.launches;
    if (total_ms) *total_ms = a.ms;
    if (total_bytes) *total_bytes = a.bytes;
    return SLOS_OK;
}

}  // extern "C"
