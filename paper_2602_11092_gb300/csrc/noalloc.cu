// Forward pass that allocates nothing and needs no caller workspace.
//
// Some callers cannot allocate device memory: a plugin running inside a host
// application whose memory pool owns every device allocation, or a
// latency-critical loop where a cudaMalloc (which may synchronise the device)
// is not acceptable.  slos_forward_noalloc serves them with a scratch buffer
// that is part of the library image: a file-scope __device__ array of
// kNoAllocScratchBytes that every GPU loading the library holds until the
// process exits.  The caller still owns U and the output.
//
// Host code cannot use the array's name as a device address (on the host it
// is only a stand-in symbol), so the device address is looked up with
// cudaGetSymbolAddress, once per device, the first time the entry point runs
// on that device (with that device current).  That first call should come
// before any stream capture.  All calls share the one array and it keeps the
// last call's contents; calls whose work overlaps on the GPU (concurrent
// streams, or several host threads) race on it and must be serialised by the
// caller.  The forward pass writes every scratch element it reads except its
// work-queue counters, which it zeroes itself at the start of every call.
//
// Device rule: the plan, U and out must all belong to the device that is
// current when the entry point is called (the scratch address is that
// device's); anything else is rejected with SLOS_ERR_INVALID_ARG.  The cached
// address stays valid for the life of the process's context on that device:
// after a cudaDeviceReset the entry point must not be called again in the
// same process.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/slos.h"
#include "plan.h"

namespace slos {
slos_status_t fail(slos_status_t st, const std::string &msg);
}

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB per device

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void *g_addr[64] = {nullptr};

slos_status_t scratch_address(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return slos::fail(SLOS_ERR_CUDA, std::string("slos_forward_noalloc: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return slos::fail(SLOS_ERR_UNSUPPORTED, "slos_forward_noalloc: device index >= 64");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return slos::fail(SLOS_ERR_CUDA, std::string("slos_forward_noalloc: cudaGetSymbolAddress failed: ") +
                                                 cudaGetErrorString(e));
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return SLOS_OK;
}

}  // namespace

extern "C" {

size_t slos_noalloc_scratch_bytes(void) { return kNoAllocScratchBytes; }

slos_status_t slos_forward_noalloc(slos_plan_t plan, const void *U, int batch, slos_output_t output, void *out,
                                   void *stream) {
    if (!plan) return slos::fail(SLOS_ERR_INVALID_ARG, "slos_forward_noalloc: NULL plan");
    size_t need = 0;
    slos_status_t st = slos_workspace_bytes(plan, batch, 0, &need);
    if (st != SLOS_OK) return st;
    if (need > kNoAllocScratchBytes)
        return slos::fail(SLOS_ERR_UNSUPPORTED,
                          "slos_forward_noalloc: this batch needs " + std::to_string(need) +
                              " bytes of scratch but the built-in scratch holds " +
                              std::to_string(kNoAllocScratchBytes) +
                              "; use a smaller batch or slos_forward with a caller workspace");
    if (batch > 0) {
        int dev = -1;
        if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->device)
            return slos::fail(SLOS_ERR_INVALID_ARG, "slos_forward_noalloc: the plan was built on device " +
                                                        std::to_string(plan->device) + ", not the current device");
        const void *ptrs[2] = {U, out};
        for (const void *q : ptrs) {
            cudaPointerAttributes at;
            if (!q || cudaPointerGetAttributes(&at, q) != cudaSuccess ||
                (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev) {
                cudaGetLastError();  // clear a sticky lookup error, if any
                return slos::fail(SLOS_ERR_INVALID_ARG,
                                  "slos_forward_noalloc: U and out must be device memory of the current device");
            }
        }
    }
    void *scratch = nullptr;
    st = scratch_address(&scratch);
    if (st != SLOS_OK) return st;
    return slos_forward(plan, U, batch, output, out, 0, scratch, kNoAllocScratchBytes, stream);
}

}  // extern "C"
