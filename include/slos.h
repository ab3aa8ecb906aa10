/*
 * libslos — batched strong simulation of linear-optical layers on one GPU.
 *
 * C ABI.  Plain pointers and sizes only; no framework types.  Every device
 * pointer is owned by the caller (allocate it however you like); a plan owns
 * only its small device-side status word.  Every call that takes a `stream`
 * (a cudaStream_t passed as void*, NULL = legacy default stream) is
 * asynchronous on that stream, allocates nothing and does not synchronise, so
 * it can be captured in a CUDA graph.  A plan additionally owns its transition
 * tables (allocated and filled once by slos_plan).  Errors are returned as status codes and
 * never thrown; `slos_last_error()` gives a message for the calling thread.
 *
 * Physics (Sec. II-A.1 "Essentials of linear optics"): an n-photon Fock state
 * |s> = |s_1..s_m> over m modes evolves through an m x m unitary U; the
 * amplitude of output Fock state t is
 *      <t|U|s> = Per(U[rows(t), cols(s)]) / sqrt(prod_j t_j! prod_i s_i!),
 * and there are C(m+n-1, n) output states.  The library computes all of them
 * at once by the photon-by-photon recursion of Sec. II-A.2/II-A.3 (SLOS): with
 * the input photons in modes c_1 <= ... <= c_n,
 *      a_0 = 1 on the vacuum,
 *      a_k(t) = sum_{j : t_j > 0} U[j, c_k] * a_{k-1}(t - e_j),
 * so a_n(t) = Per(...)/prod t_j!, p(t) = |a_n(t)|^2 prod t_j! / prod s_i!.
 *
 * Conventions used by every call:
 *   complex64  interleaved (re, im) float32.
 *   U          complex64 [batch][m][m] row-major, U[b][j][i] = U_{j,i}: input
 *              mode i is mapped to sum_j U_{j,i} |j>.
 *   outputs    index of Fock state t = its position in descending
 *              lexicographic order over compositions of n into m parts
 *              (first (n,0,...,0), last (0,...,0,n)).
 *   threshold  outcome b = set of occupied modes, 1 <= |b| <= min(n, m),
 *              ordered by |b| ascending then by colex rank of the subset;
 *              q(b) = sum of p(t) over t whose occupied set is b.
 *   gradients  PyTorch convention for complex tensors:
 *              dZ = dL/dRe Z + i dL/dIm Z.
 *   limits     2 <= m <= 24, 1 <= n <= 12, C(m+n-1, n) < 2^31; larger
 *              problems return SLOS_ERR_UNSUPPORTED.
 */
#ifndef SLOS_H
#define SLOS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct slos_plan_s *slos_plan_t;

typedef enum {
    SLOS_OK = 0,
    SLOS_ERR_INVALID_ARG = 1,
    SLOS_ERR_UNSUPPORTED = 2,
    SLOS_ERR_OOM = 3,
    SLOS_ERR_CUDA = 4,
    SLOS_ERR_TIMEOUT = 5,
    SLOS_ERR_INTERNAL = 6
} slos_status_t;

typedef enum { SLOS_DETECT_PNR = 0, SLOS_DETECT_THRESHOLD = 1 } slos_detection_t;
typedef enum { SLOS_OUT_PROBS = 0, SLOS_OUT_AMPS = 1 } slos_output_t;
/* Computation space (Sec. II-A.3, QuantumLayer): the Hilbert subspace the
 * state is represented on.  FOCK: every composition of n photons over m
 * modes.  UNBUNCHED: only collision-free states (at most one photon per
 * mode), C(m, n) of them; the recursion then runs over collision-free
 * intermediate states only, which gives the exact amplitudes of the
 * collision-free outputs (every path to such an output passes only through
 * collision-free states).  Unbunched outputs are ordered like the Fock
 * outputs restricted to them: descending lexicographic order of the
 * occupation vectors, i.e. ascending lexicographic order of the occupied-mode
 * tuples. */
typedef enum { SLOS_SPACE_FOCK = 0, SLOS_SPACE_UNBUNCHED = 1 } slos_space_t;

/* Message describing the last error on the calling thread ("" if none). */
const char *slos_last_error(void);

/* Library version string. */
const char *slos_version(void);

/* ----------------------------------------------------------------------
 * Interferometer mesh -> unitary (Sec. II-A.3: trainable parameters are the
 * phases of the physical components; Sec. II-C.1: U(x, theta) =
 * W2(theta2) S(x) W1(theta1) with data phases between two trainable
 * interferometers).
 *
 * Mesh: rectangular (Clements) layout of m columns; column c holds a
 * Mach-Zehnder interferometer on modes (k, k+1) for k = c mod 2, c mod 2 + 2,
 * ..., k <= m-2: m(m-1)/2 MZIs, P = m(m-1) phases.  MZI(theta, phi) =
 * B diag(e^{i theta}, 1) B diag(e^{i phi}, 1) with B = [[1, i], [i, 1]]/sqrt 2.
 * Phases are ordered column by column, k ascending, (theta, phi) per MZI;
 * U = T_last ... T_first.  If n_data > 0 the data screen
 * diag(e^{i x_0}, ..., e^{i x_{n_data-1}}, 1, ...) sits after the first
 * `data_col` columns (0 <= data_col <= m).
 * ---------------------------------------------------------------------- */
typedef struct {
    int m;        /* modes, 2..24 */
    int n_data;   /* data phases, 0..m, on modes 0..n_data-1 */
    int data_col; /* number of mesh columns before the data screen */
} slos_mesh_desc_t;

/* theta: float32 device [batch][m(m-1)] with row stride theta_stride_b
 *        floats (0 = one phase vector shared by the whole batch).
 * data:  float32 device [batch][n_data] with row stride data_stride_b
 *        (NULL allowed when n_data == 0).
 * U:     complex64 device [batch][m][m], fully written. */
slos_status_t mesh_unitary(const slos_mesh_desc_t *desc, const float *theta, int64_t theta_stride_b,
                           const float *data, int64_t data_stride_b, int batch, void *U, void *stream);

/* Scratch bytes needed by mesh_unitary_backward for this shape. */
slos_status_t mesh_unitary_backward_workspace(const slos_mesh_desc_t *desc, int batch,
                                              int64_t theta_stride_b, size_t *bytes);

/* Reverse sweep through the mesh.  dU: complex64 device [batch][m][m].
 * dtheta: float32 device; [m(m-1)] (summed over the batch, in a fixed order)
 * when theta_stride_b == 0, otherwise [batch][m(m-1)].  ddata: float32 device
 * [batch][n_data] (NULL allowed when n_data == 0).  Both outputs are
 * overwritten.  workspace: device scratch of the size reported above (may be
 * NULL when that size is 0). */
slos_status_t mesh_unitary_backward(const slos_mesh_desc_t *desc, const float *theta, int64_t theta_stride_b,
                                    const float *data, int64_t data_stride_b, int batch, const void *dU,
                                    float *dtheta, float *ddata, void *workspace, size_t workspace_bytes,
                                    void *stream);

/* ----------------------------------------------------------------------
 * Plans (Sec. II-A.3: the transition structure between photon-number
 * layers depends only on the input state and is built once; only the
 * U-dependent coefficients change per call).
 * ---------------------------------------------------------------------- */

/* Build a plan for input Fock state `input_state` (host, m ints summing to n).
 * mem_budget_bytes: per-instance budget (bytes) for the intermediate
 * photon-number layers 1..n-1 that slos_forward(save_for_backward=1) keeps
 * for slos_backward; 0 = keep them all.  With a budget, only layers n-1,
 * n-1-s, n-1-2s, ... are kept (s as small as fits, counting one recompute
 * segment) and the others are recomputed in the backward pass; the final
 * layer a_n is always kept.  Allocates a 64-byte device status word on the
 * current device. */
/* The same mesh with data phases formed from features and weights (the
 * angle encoding of Sec. II-C.1, phi_j = x_j * w_j): x float32 device
 * [batch][n_data] with row stride x_stride_b, w float32 device [n_data]
 * (shared by the batch).  Otherwise as mesh_unitary. */
slos_status_t mesh_unitary_weighted(const slos_mesh_desc_t *desc, const float *theta, int64_t theta_stride_b,
                                    const float *x, int64_t x_stride_b, const float *w, int batch, void *U,
                                    void *stream);

/* Reverse sweep of mesh_unitary_weighted: dtheta as in mesh_unitary_backward;
 * dx float32 device [batch][n_data] = dL/dphi_j * w_j; dw float32 device
 * [batch][n_data] (per instance, the caller sums over the batch) =
 * dL/dphi_j * x_j, or NULL when not needed.  Same workspace as
 * mesh_unitary_backward. */
slos_status_t mesh_unitary_weighted_backward(const slos_mesh_desc_t *desc, const float *theta, int64_t theta_stride_b,
                                             const float *x, int64_t x_stride_b, const float *w, int batch,
                                             const void *dU, float *dtheta, float *dx, float *dw, void *workspace,
                                             size_t workspace_bytes, void *stream);

/* Sum of per-instance gradient rows over the batch: out[p] = sum_b rows[b][p]
 * for rows float32 device [batch][width] (row stride width), out float32
 * device [width].  The chain rule for parameters every instance shares (the
 * trainable phases of Sec. II-A.3, the encoding weights w of Sec. II-C.1),
 * e.g. the per-instance dw of mesh_unitary_weighted_backward.  The order of
 * the additions is fixed (the result does not depend on the launch); batch = 0
 * writes zeros.  Returns SLOS_ERR_INVALID_ARG for NULL pointers or negative
 * sizes. */
slos_status_t mesh_sum_rows(const float *rows, int batch, int width, float *out, void *stream);

slos_status_t slos_plan(int m, int n, const int *input_state, slos_detection_t detection,
                        size_t mem_budget_bytes, slos_plan_t *out);

/* slos_plan on a chosen computation space.  SLOS_SPACE_UNBUNCHED needs PNR
 * detection and n <= m, and a plan small enough for transition tables
 * (otherwise SLOS_ERR_UNSUPPORTED); the input state may itself be bunched.
 * slos_plan(...) is slos_plan_space(..., SLOS_SPACE_FOCK, ...). */
slos_status_t slos_plan_space(int m, int n, const int *input_state, slos_detection_t detection, slos_space_t space,
                              size_t mem_budget_bytes, slos_plan_t *out);

/* n_outputs: values per instance written by slos_forward (PNR: C(m+n-1, n);
 * unbunched: C(m, n); threshold: sum_{k=1}^{min(n,m)} C(m, k)).  fock_dim:
 * number of states of the plan's space, C(m+n-1, n) or C(m, n).
 * checkpoint_stride: the s chosen from the budget (1 = every layer kept). */
slos_status_t slos_plan_query(slos_plan_t plan, int64_t *n_outputs, int64_t *fock_dim, int *checkpoint_stride);

/* Device scratch bytes that slos_forward / slos_backward need for `batch`
 * instances.  training = 0: forward only; training = 1: forward with
 * save_for_backward and the matching backward (same buffer for both). */
slos_status_t slos_workspace_bytes(slos_plan_t plan, int batch, int training, size_t *bytes);

/* Forward pass for a batch of unitaries (all with this plan's m, n, input).
 * out: PNR + SLOS_OUT_PROBS  -> float32 [batch][n_outputs] probabilities;
 *      PNR + SLOS_OUT_AMPS   -> complex64 [batch][n_outputs] amplitudes <t|U|s>;
 *      threshold (PROBS only) -> float32 [batch][n_outputs] q(b), each one sum
 *      over the pattern's states in a fixed order (outputs reproducible bit
 *      for bit; every output element is written, so out needs no clearing).
 * save_for_backward = 1 keeps the activations slos_backward needs inside
 * `workspace` (sized with training = 1); the caller must hand the same
 * workspace, untouched, to slos_backward.  The workspace must start on a
 * 256-byte boundary (as cudaMalloc and PyTorch allocations do); otherwise the
 * call returns SLOS_ERR_INVALID_ARG before any launch. */
slos_status_t slos_forward(slos_plan_t plan, const void *U, int batch, slos_output_t output, void *out,
                           int save_for_backward, void *workspace, size_t workspace_bytes, void *stream);

/* Backward pass.  dout: gradient of the loss w.r.t. slos_forward's output,
 * float32 (probabilities / threshold) or complex64 (amplitudes), row stride
 * dout_stride_b elements between instances (0 = the same row for every
 * instance).  dU: complex64 device [batch][m][m], fully overwritten
 * (columns of modes without input photons are zero). */
slos_status_t slos_backward(slos_plan_t plan, const void *U, int batch, slos_output_t output, const void *dout,
                            int64_t dout_stride_b, void *dU, void *workspace, size_t workspace_bytes, void *stream);

/* ----------------------------------------------------------------------
 * Measurement strategies on top of the output distribution (Sec. II-A.3,
 * QuantumLayer: full distribution, per-mode photon-number expectations) and
 * renormalisation onto the plan's space.  They read and write caller buffers
 * only; each has its backward.  Plans built without transition tables (the
 * largest Fock spaces) return SLOS_ERR_UNSUPPORTED for the expectations.
 * ---------------------------------------------------------------------- */

/* out[b][j] = sum_t occ_j(t) probs[b][t] over the plan's n_outputs values:
 * PNR outputs: occ_j(t) = t_j, the mean photon number in mode j; threshold
 * outcomes: occ_j(b) = [j in b], the click probability of detector j.
 * probs: float32 [batch][n_outputs]; out: float32 [batch][m].  Each value is
 * one fixed-order sum (reproducible run to run). */
slos_status_t slos_expectations(slos_plan_t plan, const float *probs, int batch, float *out, void *stream);

/* dprobs[b][t] = sum_j occ_j(t) dout[b][j]; dout float32 [batch][m],
 * dprobs float32 [batch][n_outputs] (overwritten). */
slos_status_t slos_expectations_backward(slos_plan_t plan, const float *dout, int batch, float *dprobs,
                                         void *stream);

/* Z[b] = sum_t p[b][t], q[b][t] = p[b][t] / Z[b] (the distribution
 * conditioned on the plan's space, e.g. on collision-free outcomes).  p, q:
 * float32 [batch][n_outputs] (q may be p); Z: float32 [batch]. */
slos_status_t slos_renormalise(slos_plan_t plan, const float *p, int batch, float *q, float *Z, void *stream);

/* dp[b][t] = (dq[b][t] - sum_s dq[b][s] q[b][s]) / Z[b]; dp may be dq. */
slos_status_t slos_renormalise_backward(slos_plan_t plan, const float *q, const float *Z, const float *dq, int batch,
                                        float *dp, void *stream);

/* ----------------------------------------------------------------------
 * Shot sampling (the hardware-aware design section: a photonic processor
 * returns a finite number of shots, MerlinProcessor's nsample).  Each shot
 * turns one caller-supplied uniform draw u in [0, 1) into an outcome index by
 * inverting the cumulative distribution in exact integer arithmetic: weights
 * P(t) = floor(p(t) 2^32), C(t) = P(0) + ... + P(t), T = C(n_outputs - 1);
 * the outcome is the first t with C(t) > floor(floor(u 2^32) T / 2^32).
 * Draws outside [0, 1) are clamped into it (NaN counts as 0); NaN or negative
 * weights count as 0; outcomes whose weight rounds to zero are never drawn; a
 * distribution with no weight gives -1.  The result depends on nothing but p
 * and u, bit for bit.
 * ---------------------------------------------------------------------- */

/* Device scratch bytes slos_sample needs for `batch` distributions. */
slos_status_t slos_sample_workspace_bytes(slos_plan_t plan, int batch, size_t *bytes);

/* probs: float32 [batch][n_outputs] (any non-negative weights: the
 * distribution is T-normalised); uniforms: float32 [batch][shots];
 * samples: int32 [batch][shots] outcome indices; counts: NULL or int32
 * [batch][n_outputs], overwritten with the number of shots per outcome. */
slos_status_t slos_sample(slos_plan_t plan, const float *probs, int batch, int shots, const float *uniforms,
                          int32_t *samples, int32_t *counts, void *workspace, size_t workspace_bytes, void *stream);

/* ----------------------------------------------------------------------
 * Fidelity kernel (kernel-methods section): the embedding |phi(x)> =
 * U(x)|s> of a Fock input s gives K[i][j] = |<phi_a(i)|phi_b(j)>|^2 =
 * |<s|Ua[i]^dag Ub[j]|s>|^2 = |Per(W_ij)|^2 / (prod s_i!)^2, W_ij the n x n
 * block of Ua[i]^dag Ub[j] on the photon columns.  Ua: complex64 [Na][m][m],
 * Ub: complex64 [Nb][m][m] (e.g. from mesh_unitary); K: float32 [Na][Nb].
 * W in FP32; the permanent (Glynn, Gray-code order) in double-float
 * arithmetic on the FP32 pipe (pairs of floats, about 44 bits), no FP64
 * instruction.  1 <= n <= 8
 * photons, m <= 24; otherwise SLOS_ERR_UNSUPPORTED.
 * ---------------------------------------------------------------------- */
slos_status_t slos_fidelity_kernel(int m, const int *input_state, const void *Ua, int Na, const void *Ub, int Nb,
                                   float *K, void *stream);

/* ----------------------------------------------------------------------
 * Amplitude-encoded input (Sec. II-C, amplitude encoding): the input is a
 * state vector |x> = sum_s x_s |s> over the plan's output basis (same order,
 * n photons; Fock or collision-free space) and the output is U|x>:
 *     psi(t) = sum_s <t|U|s> x_s.
 * The call builds the n-photon transfer matrix of U (K x K) layer by layer
 * with the photon-by-photon recursion, in the workspace, then applies it to
 * the batch's vectors with one complex GEMM.  One U for the whole batch.
 * PNR plans with K <= 32768 outputs (tables built at plan time); forward only.
 * ---------------------------------------------------------------------- */

/* Device scratch bytes slos_encoded_forward needs (K^2 + F_{n-1}^2 complex64). */
slos_status_t slos_encoded_workspace_bytes(slos_plan_t plan, size_t *bytes);

/* U: complex64 [m][m]; X: complex64 [batch][n_outputs] input amplitudes;
 * out: complex64 [batch][n_outputs] amplitudes (SLOS_OUT_AMPS) or float32
 * probabilities |psi(t)|^2 (SLOS_OUT_PROBS). */
slos_status_t slos_encoded_forward(slos_plan_t plan, const void *U, const void *X, int batch, slos_output_t output,
                                   void *out, void *workspace, size_t workspace_bytes, void *stream);

/* Launch-shape autotuner of a single-shape plan for one batch size (the
 * paper has no counterpart; the recursion it times is the one of Sec.
 * II-A.2).  Times a training pair (slos_forward with activations saved, then
 * slos_backward with the shared output gradient dout_shared float32 [n_outputs])
 * for each candidate launch shape: the number L of leading layers run on chip
 * (none, or 2 up to the largest that fits), the instances per CTA of those
 * launches, and the blocks per SM of the forward and backward layer grids; the
 * fastest is kept in the plan.  U, out (float32 [batch][n_outputs]), dU and
 * workspace (the training size for `batch`) are the caller's, as for
 * slos_forward / slos_backward, and are overwritten.  cache_path (may be
 * NULL): a JSON-lines file keyed by device name, plan shape and batch; a
 * cached entry is applied without timing, a new result is appended.  Call it
 * before a forward / backward pair, not between the two.  Synchronises
 * `stream`; not for stream capture. */
slos_status_t slos_autotune(slos_plan_t plan, const void *U, int batch, void *out, const float *dout_shared, void *dU,
                            void *workspace, size_t workspace_bytes, const char *cache_path, void *stream);

/* The launch shapes a plan uses: prefix_layers = L (0: none), prefix_ni,
 * fwd_blocks_per_sm, bwd_blocks_per_sm (0: the defaults, before tuning).
 * Any pointer may be NULL. */
slos_status_t slos_plan_tuning(slos_plan_t plan, int *prefix_layers, int *prefix_ni, int *fwd_blocks_per_sm,
                               int *bwd_blocks_per_sm);

/* Reads the plan's device status word (waits for `stream`), clears it, and
 * returns SLOS_ERR_TIMEOUT / SLOS_ERR_INTERNAL if a kernel reported one. */
slos_status_t slos_sync_status(slos_plan_t plan, void *stream);

slos_status_t slos_plan_destroy(slos_plan_t plan);

/* ----------------------------------------------------------------------
 * Uneven batches: instances with different (m, n, input, detection) in one
 * persistent launch.  Instances are packed: U of instance i is complex64
 * [m_i][m_i] at element offset u_offset[i]; its output is float32 [K_i] at
 * element offset out_offset[i] (PNR: probabilities, threshold: q(b)).
 * ---------------------------------------------------------------------- */
slos_status_t slos_batched_plan(int count, const int *m, const int *n, const int *const *input_states,
                                const slos_detection_t *detection, slos_plan_t *out);

/* u_offsets / out_offsets: host arrays of count + 1 int64 (the last entry is
 * the total).  workspace_bytes: device scratch for slos_batched_forward. */
slos_status_t slos_batched_query(slos_plan_t plan, int64_t *u_offsets, int64_t *out_offsets,
                                 size_t *workspace_bytes);

/* One launch of a persistent kernel over every (instance, layer, tile) work
 * item; graph-capturable.  Waits between layers are bounded: a wait that runs
 * out sets the plan's status word (read it with slos_sync_status). */
slos_status_t slos_batched_forward(slos_plan_t plan, const void *U_packed, float *out_packed, void *workspace,
                                   size_t workspace_bytes, void *stream);

/* Fault injection for tests of the bounded waits: while enabled, every
 * slos_batched_forward launch starts one layer's completion counter so that
 * it never completes and shortens the wait limit to about a millisecond; the
 * items waiting on it give up, the launch ends, and slos_sync_status returns
 * SLOS_ERR_TIMEOUT.  No fault, trap or hang is involved. */
slos_status_t slos_batched_inject_stall(slos_plan_t plan, int enable);

/* Times the launch configurations of slos_batched_forward on this GPU and
 * keeps the fastest in the plan; results are cached in the JSON file
 * `cache_path` (NULL = no cache), keyed by device name and problem shape. */
slos_status_t slos_batched_autotune(slos_plan_t plan, const void *U_packed, float *out_packed, void *workspace,
                                    size_t workspace_bytes, const char *cache_path, void *stream);

/* ----------------------------------------------------------------------
 * Index arithmetic, exposed for exact (bit-for-bit) testing.
 * ---------------------------------------------------------------------- */

/* Host: rank of composition t (m ints summing to k) in descending-lex order. */
int64_t slos_host_rank(int m, const int *t);
/* Host: inverse of slos_host_rank; writes m ints. */
slos_status_t slos_host_unrank(int m, int k, int64_t rank, int *t);

/* Host: the transition graph of layer k (Sec. II-A.3) that plans build
 * once and reuse.  rowptr: int32 [C(m+k-1,k) + 1]; entries: uint32
 * [m * C(m+k-2,k-1)], child c owns entries rowptr[c] .. rowptr[c+1]-1, each
 * (parent rank << 6) | (mode << 1) | last; ctab: int32 [C(m+k-2,k-1)][m],
 * ctab[c'][j] = rank_k(t' + e_j).  Host buffers owned by the caller; any may
 * be NULL.  SLOS_ERR_UNSUPPORTED when parent ranks do not fit 26 bits. */
slos_status_t slos_host_transition_table(int m, int k, int32_t *rowptr, uint32_t *entries, int32_t *ctab);

/* Host: the split-lattice tables that plans of 8..16 modes build once for
 * their backward layers (Sec. II-A.3's transition graph regrouped by head
 * blocks).  The m modes are split into head modes 0..h-1 and tail modes
 * h..m-1; the states of a layer with the same head occupations form one
 * block of consecutive ranks.  Layer k (2 <= k <= n), whose parents are the
 * states of layer k-1:
 *   counts   int64 [2]: blocks, chunks (always written).
 *   bdesc    int32 [blocks][4]: the blocks of layer k-1: base rank, size, base
 *            rank of the same head in layer k, tail photons.
 *   bhead    int32 [blocks][8]: base rank in layer k of head t_H + e_j, j < h,
 *            then 0.
 *   bchunk   int32 [chunks]: block holding state 4 * chunk of layer k-1.
 * Any array may be NULL.  h: head modes (written).  SLOS_ERR_UNSUPPORTED
 * when the plan shape takes no split tables. */
slos_status_t slos_host_split_layer(int m, int n, int k, int *h, int64_t *counts, int32_t *bdesc, int32_t *bhead,
                                    int32_t *bchunk);

/* Host: the tail child table of the split lattice over the m - h tail modes,
 * for tail photon numbers rho = 0..n-1.  offsets int32 [n+1]: start of rho's
 * child rows (rows of 8; offsets[n] = the row count).  count: child entries
 * (always written).  ctab: uint16 local position of t_L + e_j within the
 * tail lattice of rho + 1 photons for j < m - h, then 0.  Any array may be
 * NULL. */
slos_status_t slos_host_split_tail(int m, int n, int *h, int32_t *offsets, int64_t *count, uint16_t *ctab);

/* Host: range check of a layer's transition tables as plans upload them
 * (every plan runs it before uploading).  slots: uint32 [C(m+k-1,k)][kw],
 * each (parent rank << 5) | mode for an occupied mode, or 24 (padding); every
 * state needs at least one parent.  ctab: int32 [C(m+k-2,k-1)][m] child
 * ranks.  SLOS_ERR_INTERNAL, naming the first bad entry, when an index is out
 * of range. */
slos_status_t slos_host_validate_tables(int m, int k, int kw, const uint32_t *slots, const int32_t *ctab);

/* Host-side fault injection for tests; it makes host calls fail the way the
 * real failure would, so no GPU is faulted.  SLOS_INJECT_ALLOC_FAIL: the
 * value-th device allocation made while building plans from now on fails as
 * out of memory (one shot; 0 = off).  SLOS_INJECT_STREAM_DEVICE: the device
 * of any stream passed to slos_forward / slos_backward is reported as
 * `value` (-1 = off), so a plan used with another device's stream is
 * exercised; such calls return SLOS_ERR_INVALID_ARG before any launch.
 * SLOS_INJECT_TABLE_BUDGET: while value != 0, every plan built finds its
 * transition tables over the per-plan table budget, as plans too large for
 * tables do, and so takes the arithmetic-index kernels (no tables, no split
 * lattice, no on-chip forward); plans keep the mode they were built in.
 * SLOS_INJECT_NONE clears all three. */
typedef enum {
    SLOS_INJECT_NONE = 0,
    SLOS_INJECT_ALLOC_FAIL = 1,
    SLOS_INJECT_STREAM_DEVICE = 2,
    SLOS_INJECT_TABLE_BUDGET = 3
} slos_inject_t;
slos_status_t slos_inject_fault(slos_inject_t kind, int value);

/* Device: for ranks [first, first + count) of layer k (k photons, m modes)
 * write the composition (uint8 [count][m]) and the parent index
 * rank_{k-1}(t - e_j) for every mode j (int32 [count][m], -1 where t_j = 0),
 * computed by the same device code the SLOS kernels use.  Either output may
 * be NULL. */
slos_status_t slos_device_index_table(int m, int k, int64_t first, int64_t count, uint8_t *compositions,
                                      int32_t *parents, void *stream);


/* ----------------------------------------------------------------------
 * Tracing.  Every kernel the library launches increments a process-wide
 * counter.  With profiling enabled, each launch is also bracketed by two CUDA
 * events recorded on its own stream and tagged with a name and the number of
 * algorithmic bytes the launch moves (layered model: every photon-number
 * layer written once and read once, complex64 amplitudes, float32
 * probabilities).  Do not enable it while capturing a CUDA graph.
 * ---------------------------------------------------------------------- */
slos_status_t slos_profile_enable(int enable);
/* Drops every recorded launch and resets the launch counter. */
slos_status_t slos_profile_reset(void);
/* Kernels launched since the last reset (counted with or without profiling). */
int64_t slos_launch_count(void);
/* Waits for the recorded events and aggregates them by name.  Returns the
 * number of distinct names; entry i (0 <= i < count) is read with
 * slos_profile_entry. */
int slos_profile_collect(void);
slos_status_t slos_profile_entry(int i, char *name, size_t name_len, int64_t *launches, double *total_ms,
                                 double *total_bytes);

/* ----------------------------------------------------------------------
 * Allocation-free forward pass.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory themselves,
 * such as a plugin inside a host application whose memory pool owns all
 * device allocations, or a latency-critical loop that must never wait on a
 * cudaMalloc.
 *
 * Same computation and output as slos_forward(plan, U, batch, output, out,
 * save_for_backward = 0, ...), but the intermediate photon-number layers live
 * in a scratch array built into the library (slos_noalloc_scratch_bytes(),
 * 32 MiB, held by every GPU that loads the library until the process exits).
 * The caller still passes U and out.  Calls no cudaMalloc / cudaFree.
 *
 * - Returns SLOS_ERR_UNSUPPORTED, with a message naming both sizes, when the
 *   batch needs more scratch than that (slos_workspace_bytes(plan, batch, 0)).
 * - The first call on a device looks up the array's device address with that
 *   device current; make that first call before any stream capture.
 * - Every call uses the same array: calls that overlap on the GPU (different
 *   streams, or several host threads) race and must be serialised by the
 *   caller.  No state carries over between calls (the call zeroes the few
 *   counters it needs).
 * - The plan, U and out must belong to the current device; otherwise
 *   SLOS_ERR_INVALID_ARG.  The looked-up address is kept for the process: do
 *   not call this entry point again on a device after cudaDeviceReset.
 * ---------------------------------------------------------------------- */
size_t slos_noalloc_scratch_bytes(void);
slos_status_t slos_forward_noalloc(slos_plan_t plan, const void *U, int batch, slos_output_t output, void *out,
                                   void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SLOS_H */
