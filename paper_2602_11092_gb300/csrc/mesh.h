// Internal launch interface of the mesh kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace slos {

struct MeshArgs {
    const float *theta;
    int64_t theta_stride;
    const float *data;
    int64_t data_stride;
    const float *data_w;  // per-mode weights: phase j = data_j * data_w[j] (null: the data are the phases)
    float2 *U;
    int m, n_data, data_col, B;
};

struct MeshBwdArgs {
    const float *theta;
    int64_t theta_stride;
    const float *data;
    int64_t data_stride;
    const float *data_w;  // as in MeshArgs
    float *dw;            // [B][n_data] per-instance gradient of the weights (may be null)
    const float2 *dU;
    float *dtheta;     // [B][P] (per instance)
    int64_t dtheta_stride;
    float *ddata;      // [B][n_data]
    int m, n_data, data_col, B;
};

cudaError_t mesh_forward_launch(const MeshArgs &a, cudaStream_t s);
// dtheta_shared != null: a.dtheta holds per-instance rows, summed into it.
cudaError_t mesh_backward_launch(const MeshBwdArgs &a, float *dtheta_shared, cudaStream_t s);
// out[p] = sum over rows b < B of part[b][p] (rows of P floats), fixed order.
cudaError_t mesh_sum_rows_launch(const float *part, int B, int P, float *out, cudaStream_t s);

}  // namespace slos
