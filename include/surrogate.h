/*
 * libslos — learned surrogate of a photonic layer (BF16 MLP on the tensor
 * cores), trained on distributions the exact simulator produces.
 *
 * The differentiable layers of the paper (Sec. II-A.3, II-B) map phases to an
 * output distribution; this model approximates that map for one fixed layer
 * (here the m=12, n=6 layer): features [sin phi, cos phi] -> n_hidden GELU
 * layers of width `hidden` -> logits over the n_outputs Fock states ->
 * softmax.  It is trained with the KL divergence KL(p_exact || q); the exact
 * path (slos_forward) stays the arbiter of its total-variation error and the
 * fallback for samples that fail the check.
 *
 * Conventions: all pointers are device pointers owned by the caller unless
 * stated otherwise; a model owns its weights, Adam moments and activation
 * buffers (allocated once by surr_create for batches up to max_batch, so the
 * forward and training calls allocate nothing).  Every call is asynchronous
 * on `stream` (cudaStream_t as void*); errors are status codes with a message
 * from slos_last_error().
 */
#ifndef SLOS_SURROGATE_H
#define SLOS_SURROGATE_H

#include <stddef.h>
#include <stdint.h>

#include "slos.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct surr_model_s *surr_model_t;

/* Tensor-core GEMM (tcgen05 + TMA + TMEM): C[M][N] = A[M][K] . B[N][K]^T with
 * A, B BF16 row-major (row strides lda, ldb elements; K, lda, ldb multiples
 * of 8; 16-byte aligned), FP32 accumulation.  Epilogue `epi`:
 *   0: C = acc (float [M][ldc])          1: C = acc + bias[n] (float)
 *   2: aux = bf16(acc + bias[n]), C = bf16(gelu(aux))   (GELU, tanh form)
 *   3: C = bf16(acc * gelu'(aux))         4: C += acc (float)
 * The kernel's pipeline waits are bounded; a wait that runs out is reported
 * by surr_sync_status. */
slos_status_t surr_gemm_bf16(int epi, int M, int N, int K, const void *A, int64_t lda, const void *B, int64_t ldb,
                             void *C, int ldc, const float *bias, void *aux, void *stream);

/* Waits for `stream`, then returns SLOS_ERR_TIMEOUT (and clears the flag) if
 * a tensor-core GEMM reported a pipeline wait that ran out. */
slos_status_t surr_sync_status(void *stream);

/* Model with n_phases phase inputs (2*n_phases features), n_hidden_layers of
 * width `hidden`, n_outputs logits; weights He-uniform from `seed`, biases 0.
 * 2*n_phases, hidden, n_outputs and max_batch must be multiples of 8. */
slos_status_t surr_create(int n_phases, int hidden, int n_hidden_layers, int n_outputs, int max_batch,
                          unsigned long long seed, surr_model_t *out);
slos_status_t surr_destroy(surr_model_t model);

/* Input harmonics (0 = off, the default): with H > 0 the `phases` argument
 * of surr_forward / surr_train_step holds n_phases / H values x_j per row and
 * the model's phases are h * x_j for h = 1..H (phase index (h - 1) * n_x + j),
 * formed in the feature kernel.  H must divide n_phases.  (The data phases of
 * an angle-encoded layer enter every amplitude through e^{i x_j}, so the
 * output distribution is a trigonometric polynomial in them, Sec. II-C.1;
 * its harmonics are the natural features.) */
slos_status_t surr_set_input_harmonics(surr_model_t model, int harmonics);

/* phases: float [B][n_phases]; probs: float [B][n_outputs] = softmax(logits).
 * B a multiple of 8, <= max_batch. */
slos_status_t surr_forward(surr_model_t model, const float *phases, int B, float *probs, void *stream);

/* One Adam step (lr; beta 0.9/0.999; eps 1e-8) on the batch mean of
 * KL(target || softmax(logits)); target: float [B][n_outputs] (rows sum to 1).
 * loss_rows: float [B] per-sample KL (may be NULL). */
slos_status_t surr_train_step(surr_model_t model, const float *phases, const float *target, int B, float lr,
                              float *loss_rows, void *stream);

/* Host copies of layer `layer` (0 .. n_hidden_layers; the last is the output
 * layer): W float [fan_out][fan_in], b float [fan_out]; grads are those of
 * the last surr_train_step (before its Adam update).  Synchronous. */
slos_status_t surr_get_param(surr_model_t model, int layer, float *w_host, float *b_host);
slos_status_t surr_set_param(surr_model_t model, int layer, const float *w_host, const float *b_host);
slos_status_t surr_get_grad(surr_model_t model, int layer, float *gw_host, float *gb_host);

/* Training checkpoint and resume: writes the FP32 weights, the Adam moments
 * and step count, and a caller's data-stream position (stream_index) to the
 * file `path`; surr_load restores them into a model of the same dimensions
 * (SLOS_ERR_INVALID_ARG otherwise), so that training resumed from the file
 * repeats, bit for bit, the training that continued in memory.  Synchronous. */
slos_status_t surr_save(surr_model_t model, const char *path, int64_t stream_index);
slos_status_t surr_load(surr_model_t model, const char *path, int64_t *stream_index);

/* ---- checks used by the inference driver (exact path as arbiter) ---- */

/* tv[i] = 1/2 sum_t |q[rows[i]][t] - p[i][t]| : total variation of checked
 * rows.  q float [*][K], rows int [n], p float [n][K] (exact), tv float [n]. */
slos_status_t surr_tv_rows(const float *q, const int *rows, const float *p, int n, int K, float *tv, void *stream);

/* Cheap screen for every sample: the surrogate's mean photon number per mode,
 * sum_t q[b][t] t_j (occ: uint8 [K][m] occupations of the output states),
 * against the exact value sum_i |U[b][j][i]|^2 s_i (Sec. II-A.1); flag[b] is
 * set to 1 (never cleared) when the differences summed over the modes exceed
 * tol.  That sum is at most 2 n TV(exact, surrogate) for n photons, so with
 * tol = 2 n t a flagged sample provably has TV > t.
 * input_state: host, m ints.  marg_scratch: float [B][m]. */
slos_status_t surr_screen(const float *q, int B, int K, const uint8_t *occ, int m, const void *U, const int *input_state,
                          float tol, float *marg_scratch, int *flag, void *stream);

/* dst[rows[i]][:] = src[i][:] (K floats) and dst[i][:] = src[rows[i]][:]. */
slos_status_t surr_scatter_rows(const float *src, const int *rows, int n, int K, float *dst, void *stream);
slos_status_t surr_gather_rows(const float *src, const int *rows, int n, int W, float *dst, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SLOS_SURROGATE_H */
