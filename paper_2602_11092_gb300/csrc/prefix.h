// Launch interface of the on-chip prefix kernels (slos_prefix.cu): the first
// L photon-number layers of a table plan, forward and backward, one launch
// each, with every layer in shared memory.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace slos {

// Shared memory a prefix CTA may use, and the per-instance bound that picks L.
constexpr size_t kPrefixSmemLimit = 200 * 1024;
constexpr size_t kPrefixInstBytes = 100 * 1024;
constexpr int kPrefixMaxNI = 4;
constexpr int kPrefixThreads = 512;

struct PrefixArgs {
    const float2 *U;                          // [B][m][m]
    const uint32_t *slots[kMaxPhotons + 1];   // forward parent slots of layer k (plan tables)
    int kw[kMaxPhotons + 1];
    const int32_t *ctab[kMaxPhotons + 1];     // child table of layer k: [F_{k-1}][m], rank of t' + e_j
    int F[kMaxPhotons + 1];
    int cols[kMaxPhotons];                    // input mode of photon k (ascending)
    // forward: layer k <= L is written to out[k] (group layout [NG][F_k][32]) when non-null
    float2 *out[kMaxPhotons + 1];
    // backward: G_L (group layout) in, the dU partial row of each layer k <= L out
    const float2 *GL;
    float2 *dUpart[kMaxPhotons + 1];          // [NG][1][32][m] of layer k
    int cap[2];                               // states per instance of the even / odd layer buffers
    int asum;                                 // backward: states of a_0..a_{L-1} per instance
    int m, L, B, NI;
};

// Largest L (2 <= L <= n - 1) whose backward working set fits kPrefixInstBytes
// per instance; 0 when no prefix of two or more layers fits.
int slos_prefix_layers(int m, int n, const int64_t *F);
// Instances per CTA for a batch (1, 2 or 4).
int slos_prefix_ni(int m, int L, const int64_t *F, int batch, int sm_count);
size_t slos_prefix_fwd_smem(int NI, int L, const int64_t *F);
size_t slos_prefix_bwd_smem(int NI, int L, const int64_t *F);
cudaError_t slos_prefix_init();
cudaError_t slos_launch_prefix_fwd(const PrefixArgs &a, cudaStream_t s);
cudaError_t slos_launch_prefix_bwd(const PrefixArgs &a, cudaStream_t s);

}  // namespace slos
