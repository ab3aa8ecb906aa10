// Launch interface of the whole-plan on-chip forward (slos_fused.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace slos {

// Shared memory a fused CTA may use.
constexpr size_t kFusedSmemLimit = 200 * 1024;
// Sorted walk: the final layer is sorted by occupied modes within tiles of
// this many consecutive output indices.
constexpr int64_t kFusedOutTile = 4096;

struct FusedArgs {
    const float2 *U;                          // [B][m][m]
    void *out;                                // float [B][K] or complex64 [B][K]
    int sorted;                               // walk: 0 Fock order, 1 sorted 32-position blocks
    // Fock order
    const float *w;                           // final layer: prod t! / prod s!  [F_n]
    const uint32_t *slots[kMaxPhotons + 1];   // parent slots of layer k (plan tables)
    int kw[kMaxPhotons + 1];
    int F[kMaxPhotons + 1];
    // sorted order (tables.h, FusedLayer)
    const float *ws;                          // final layer: weight per position
    const int32_t *id;                        // final layer: output index per position, -1 padding
    const uint32_t *rows[kMaxPhotons + 1];    // layer k: slot rows of its 32-position blocks
    const uint32_t *blk[kMaxPhotons + 1];     // layer k: per block, row offset << 4 | slots
    int nblk[kMaxPhotons + 1];
    int cols[kMaxPhotons];                    // input mode of photon k (ascending)
    int cap[2];                               // states per instance in buffer 0 (even k) and 1 (odd k)
    int m, n, B, K, NI;                       // NI: instances per CTA
    int threads;                              // CTA size: 512 or 1024
};

size_t slos_fused_smem(int NI, int n, const int cap[2]);
int slos_fused_max_ni();
cudaError_t slos_fused_init();
cudaError_t slos_launch_fused(const FusedArgs &a, int epi, cudaStream_t s);

}  // namespace slos
