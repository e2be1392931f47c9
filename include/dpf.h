/*
 * dpf.h - C ABI of the GB300 look-ahead decentralized particle filter.
 *
 * The method is the look-ahead decentralized particle filter (LA-DPF) of
 * "Decentralized, Adaptive, Look-Ahead Particle Filtering" (Ahmed, Bibalan,
 * de Freitas, Fauvel; arXiv:1203.2394): an outer particle filter over the first
 * state block x with N particles, each carrying M inner particles of the second
 * block z (Section 2, eq. filteringProblem), advanced by the four steps of
 * Fig. 4 with the Monte Carlo optimal-proposal weights of eq. weightsMC.
 *
 * Conventions for every entry point:
 *  - The return value is a dpf_status; no call aborts, traps or exits.
 *  - "device" pointers are CUDA device (or managed) memory on the current
 *    device; "host" pointers are ordinary host memory. The caller owns every
 *    buffer it passes; a context owns its own device state.
 *  - "stream" is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream). Work is ordered on that stream.
 *  - On failure, dpf_last_error() returns a thread-local message.
 */
#ifndef DPF_H
#define DPF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DPF_OK = 0,
  DPF_E_INVALID = 1,     /* bad argument (null pointer, size out of range, bad model) */
  DPF_E_NOMEM = 2,       /* a device allocation failed; nothing leaked */
  DPF_E_CUDA = 3,        /* a CUDA runtime call failed */
  DPF_E_TIMEOUT = 4,     /* a bounded device-side wait gave up (the scan look-back) */
  DPF_E_NUMERIC = 5,     /* all weights zero, or a NaN weight */
  DPF_E_UNSUPPORTED = 6  /* a valid request outside the compiled configurations */
} dpf_status;

enum { DPF_F32 = 0, DPF_F64 = 1 };          /* precision / dtype codes */
enum { DPF_MODEL_CLG = 1,                  /* conditionally linear-Gaussian family */
       DPF_MODEL_PAPER1 = 2, DPF_MODEL_PAPER2 = 3 }; /* the paper's models 1 and 2 (Table 1) */
enum { DPF_SYS_GLOBAL = 0, DPF_SYS_LOCAL = 1 }; /* resampling rules, see dpf_resample */
enum { DPF_TC_TF32 = 0, DPF_TC_TF32X3 = 1, DPF_TC_BF16 = 2 }; /* tensor-core operand modes */

typedef struct dpf_ctx dpf_ctx; /* opaque; created by dpf_create, freed by dpf_destroy */

/*
 * The state-space model of eq. mainDPF (Section 2), in the conditionally
 * linear-Gaussian family, on a state s of dimension d observed through y of
 * dimension dy. With x = the first d1 coordinates of s in the order given by
 * perm and z = the remaining d2 = d - d1:
 *   x_{t+1} = g(x_t, t) + A_xx x_t + A_xz z_t + v^x
 *   z_{t+1} =             A_zx x_t + A_zz z_t + v^z      [v^x; v^z] ~ N(0, Q)
 *   y_t     = qc x_t.^2 + H_x x_t + H_z z_t + e_t        e_t ~ N(0, R)
 *   s_0 ~ N(m0, P0)
 * g(x, t) = growth[0] x + growth[1] x / (1 + x^2) + growth[2] cos(growth[3] t)
 * per coordinate when growth_x is set (the growth map of Table 1), else 0; the
 * qc x.^2 term is present when quad_obs is set (then dy must equal d1).
 * All matrices are host, row-major, in the user's coordinate order, read once
 * by dpf_create (the caller keeps ownership). Q must have no x/z cross terms
 * after the permutation; H_z Q_z H_z^T must be positive definite.
 */
typedef struct {
  int32_t kind;        /* DPF_MODEL_CLG */
  int32_t d;           /* state dimension */
  int32_t dy;          /* observation dimension */
  int32_t precision;   /* DPF_F32 or DPF_F64: the arithmetic of the step */
  int32_t growth_x;    /* 0/1 */
  int32_t quad_obs;    /* 0/1 */
  const int32_t* perm; /* d entries: internal coordinate c is user coordinate perm[c]
                          (x block first); NULL = identity */
  const double* A;     /* d x d */
  const double* Q;     /* d x d, symmetric positive definite */
  const double* H;     /* dy x d */
  const double* R;     /* dy x dy, symmetric positive definite */
  const double* m0;    /* d */
  const double* P0;    /* d x d, symmetric positive definite */
  double growth[4];
  double qc;
} dpf_model_desc;

/*
 * The paper's benchmark models (Table 1), kind DPF_MODEL_PAPER1 or DPF_MODEL_PAPER2
 * (FP32 only; the matrices, growth and qc fields are not read; d and dy must be 2 and 1
 * for model 1, 4 and 1 for model 2, with d1 = d2 = d / 2; perm may be NULL or the
 * identity, or for model 1 {1, 0}: the table's z as the outer block and its x as the
 * inner one, the second decomposition of Section 4.3; the filtered mean comes back in the
 * table's order either way):
 *   model 1: x' = x + z / (1 + z^2) + v_x, z' = x + 0.5 z + 25 z / (1 + z^2) + 8 cos(1.2 t) + v_z,
 *            y = atan(x) + z^2 / 20 + e, (v_x, v_z) ~ N(0, [[1, 0.1], [0.1, 1]]);
 *   model 2: x1' = 0.5 x1 + 8 sin t + v, x2' = 0.4 x1 + 0.5 x2 + v, z1' = z1 + z2 / (1 + z2^2) + v,
 *            z2' = z1' + 0.5 z2 + 25 z2 / (1 + z2^2) + 8 cos(1.2 t) + v,
 *            y = (x1 + x2) / (1 + x1^2) + atan(z1) + z2^2 / 20 + e, the z noises ~ N(0, [[1, 0.1], [0.1, 10]]),
 *            the x noises ~ N(0, I);
 * e ~ N(0, 1), s_0 ~ N(0, I); t in the sine and cosine is the source step of the
 * transition. The inner draws are conditioned on x_t through the noise covariance. With
 * these kinds dpf_create (L <= 32), dpf_create_pf and dpf_create_std (with
 * dpf_set_gaussian_approx) serve the models; the batched form and the learned proposal
 * do not.
 */

/*
 * Create a filter: N outer particles of the x block (d1 coordinates), each with
 * M inner particles of the z block (d2 coordinates), and L look-ahead draws per
 * outer particle (the N_x' of Fig. 4 step 1). Allocates the device state and
 * draws the initial particles (Fig. 4, "Initialize": x_0 ~ p(x_0),
 * z_0 ~ p(z_0 | x_0), equal inner weights) on `stream`.
 * Limits: 1 <= M <= 1024, 1 <= L <= 64, 1 <= N < 2^31, d1 + d2 == model->d.
 * Random numbers: Philox4x32-10 keyed by (seed, filter id 0) and counted by
 * (step, outer index, purpose | inner index, block), so results depend only on
 * the seed, not on the launch configuration.
 * Returns DPF_E_UNSUPPORTED for a (precision, d1, d2, dy) with no compiled kernel.
 * On success *out owns the state until dpf_destroy.
 */
dpf_status dpf_create(const dpf_model_desc* model, int32_t d1, int32_t d2, int64_t N, int32_t M,
                      int32_t L, uint64_t seed, void* stream, dpf_ctx** out);

/*
 * One LA-DPF step t = (number of previous steps) + 1 with observation y_t
 * (Fig. 4 steps 1-4): look-ahead draws and eq. weightsMC weights for every
 * outer particle, global systematic resampling of the outer set, selection of
 * x_t from the ancestor's look-ahead draws, local systematic resampling and
 * propagation of each inner set.
 *  y_t:         dy values of the context's precision (float or double); host
 *               memory when y_on_device == 0, device memory otherwise.
 *  out_mean:    host, d doubles, or NULL: the filtered mean E[s_t | y_1..t] in
 *               the user's coordinate order.
 *  out_logZ:    host, 1 double, or NULL: the running log-evidence estimate
 *               log p(y_1..t) (sum over steps of the outer evidence of eq. weightsopt).
 * With both outputs NULL the call only enqueues work (no synchronisation);
 * otherwise it synchronises the stream and reports device-side errors.
 */
dpf_status dpf_step(dpf_ctx* ctx, const void* y_t, int32_t y_on_device, double* out_mean,
                    double* out_logZ);

/*
 * The same step with every input and output in device memory, fully
 * stream-ordered and never synchronising: y_t (dy values of the context's
 * precision), mean_out (d doubles) and logZ_out (1 double) are device pointers;
 * either output may be NULL. Device-side errors are reported by the next
 * synchronising call (dpf_step with outputs, dpf_sync).
 */
dpf_status dpf_step_async(dpf_ctx* ctx, const void* y_t_device, double* mean_out_device,
                          double* logZ_out_device);

/* Wait for the context's stream and report any latched device-side error. */
dpf_status dpf_sync(dpf_ctx* ctx);

/*
 * Systematic resampling ("standard resampling", DPF steps 2 and 6; LA-DPF step
 * 3) in an exact integer form, so results are identical on any hardware:
 *   e = floor(log2(max W)), B = ceil(log2 n), c_i = floor(W_i 2^(S-e)),
 *   cum_i = c_0 + ... + c_i, C = cum_{n-1},
 *   out[k] = min{ i : cum_i * n * 2^b > (k * 2^b + u_b) * C },  k = 0..n-1.
 * DPF_SYS_GLOBAL: S = 62 - B, b = 32, u_b = u (128-bit products; any n < 2^31).
 * DPF_SYS_LOCAL:  S = 31 - B, b = 16, u_b = u >> 16 (64-bit; segment length <= 1024).
 *  w:       device, n_total weights of `dtype` (DPF_F32/DPF_F64), >= 0, finite,
 *           unnormalised; n_seg consecutive segments of n_total / n_seg each.
 *  n_seg:   number of segments (>= 1; must divide n_total). Each segment is
 *           resampled independently with its own uniform word u[s].
 *  u:       device, n_seg 32-bit words.
 *  out_idx: device, n_total int32 ancestor indices, local to each segment.
 * DPF_SYS_GLOBAL accepts n_seg == 1 only. A segment whose weights are all zero,
 * or any negative/NaN/infinite weight, gives DPF_E_NUMERIC (after synchronising).
 * Allocates temporary device memory for the scan state; synchronises `stream`.
 */
dpf_status dpf_resample(const void* w, int32_t dtype, int64_t n_total, int64_t n_seg, int32_t rule,
                        const uint32_t* u, int32_t* out_idx, void* stream);

/*
 * dpf_resample with DPF_SYS_GLOBAL (one segment), for callers that cannot
 * allocate device memory while they resample - for example a control loop that
 * must not allocate after start-up, or an application whose framework allocator
 * already holds the whole device. The paper has no counterpart; this is a
 * property of the library, not of the method.
 * It makes no cudaMalloc, cudaFree or other allocating call: its scratch (the
 * largest weight, the quantised total and the look-back state of the scan) is
 * a fixed device array of about 40 KB, one per device, held from the first
 * call until the process exits. Consequences:
 *  - n may be at most 4,194,304; larger n gives DPF_E_INVALID (use dpf_resample).
 *  - Every call on a device shares that array and leaves its contents behind;
 *    each call clears the part it uses first. Calls whose work overlaps on the
 *    GPU (different streams, or several host threads) race on it and give
 *    wrong indices: serialise them.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress); make that first call before any stream capture.
 * Arguments, results and errors are those of dpf_resample with n_total = n,
 * n_seg = 1 and rule = DPF_SYS_GLOBAL; it synchronises `stream`.
 */
dpf_status dpf_resample_noalloc(const void* w, int32_t dtype, int64_t n, const uint32_t* u,
                                int32_t* out_idx, void* stream);

/*
 * The library's Box-Muller transform (the normal draws of every step) applied
 * to given 32-bit words, for verifying its accuracy against the exact formula
 * n0 = sqrt(-2 ln u_a) cos(2 pi u_b), n1 = sqrt(-2 ln u_a) sin(2 pi u_b) with
 * u = ((w >> 9) + 1/2) 2^-23: out[2p] and out[2p+1] come from words[2p] (u_a)
 * and words[2p+1] (u_b). words: device, 2 n_pairs words; out: device, 2 n_pairs
 * values of `dtype` (DPF_F32 or DPF_F64, selecting the FP32 or FP64 transform).
 * Stream-ordered; does not synchronise.
 */
dpf_status dpf_box_muller(const uint32_t* words, int64_t n_pairs, int32_t dtype, void* out,
                          void* stream);

/*
 * The fifth-generation tensor-core product that the high-dimensional step
 * (A z for a 56-dimensional z block) and the learned proposal build on, run
 * alone: D = A B^T with FP32 accumulation. The paper has no counterpart; this
 * exposes the building block so that it can be checked against a plain product.
 *   mode DPF_TC_TF32:   A, B float; each operand rounded to TF32 once.
 *   mode DPF_TC_TF32X3: A, B float; each operand split as hi = tf32(v),
 *                       lo = tf32(v - hi) and D = A_lo B_hi + A_hi B_lo + A_hi B_hi
 *                       (close to an FP32 product).
 *   mode DPF_TC_BF16:   A, B bfloat16.
 * A: M x K, B: N x K, D: M x N float, all row-major device buffers owned by the
 * caller. M a multiple of 128; N a multiple of 16 in [16, 128]; K a multiple of
 * 8 up to 64 (TF32 modes) or of 16 up to 128 (BF16). Other shapes:
 * DPF_E_INVALID. Synchronises the stream; DPF_E_TIMEOUT if the MMAs did not
 * complete within the kernel's bounded wait.
 */
dpf_status dpf_tc_matmul(const void* A, const void* B, float* D, int32_t M, int32_t N, int32_t K,
                         int32_t mode, void* stream);

/* Diagnostics of the last step: outer effective sample size 1/sum W^2 (with
 * normalised W), the step counter t, and the last step's log p(y_t | y_1..t-1). */
dpf_status dpf_diag(dpf_ctx* ctx, double* ess_outer, int64_t* step, double* logZ_step);

/*
 * The bootstrap particle filter over the full state s = (x, z) (the baseline of the
 * paper's Section 4.1): N particles, each propagated from its resampled ancestor by
 * the model's transition, x_t = mu_x(x_{t-1}) + A_xz z_{t-1} + chol(Q_x) e_x and
 * z_t = A_zx x_{t-1} + A_zz z_{t-1} + chol(Q_z) e_z (e_x, e_z the Philox normals of
 * purposes 12 and 13 at counter (t, i, purpose, 0)), weighted by log N(y_t; h(s_t), R),
 * then resampled by the global systematic rule of dpf_resample. The initial particles
 * are the filter's initial draw with M = 1. Same model descriptor and variants as
 * dpf_create; the context then takes dpf_step, dpf_step_async, dpf_diag (ESS of the
 * weights), dpf_read ("x", "z": the particles of step t; "lw": their log-weights; "anc")
 * and dpf_destroy. out_mean of dpf_step is the weighted mean of step t, out_logZ the
 * cumulative log-evidence.
 */
dpf_status dpf_create_pf(const dpf_model_desc* model, int32_t d1, int32_t d2, int64_t N, uint64_t seed,
                         void* stream, dpf_ctx** out);

/*
 * The decentralized particle filter without look-ahead (Fig. dpf, the filter the LA-DPF
 * extends), with the prior as both proposals: each call t draws x_t of every outer
 * particle from the mixture prior of its ancestor's inner set (the component by the
 * one-draw local systematic rule on qbar, word (t, i, 3 = LA_J, 0); the normals of
 * (t, i, 4 = LA_X, 0)), resamples the inner set locally by qbar p(x_t | x_{t-1}, z)
 * (word (t, i, 8 = INNER, 0)), propagates it by the z prior (normals (t, i, 9 = PROP,
 * j)), weighs it by p(y_t | x_t, z_t) (qbar = the normalised weights), gives the outer
 * particle log w = log mean_j p(y_t | x_t, z_t^(j)) and resamples the outer set by the
 * global systematic rule. The initial state is the filter's initial draw. Same model
 * descriptor, variants and M limits as dpf_create (L is not used); dpf_step's out_mean is
 * the weighted mean of step t; dpf_read ("x", "z", "lq") gives the state of step t.
 */
dpf_status dpf_create_std(const dpf_model_desc* model, int32_t d1, int32_t d2, int64_t N, int32_t M,
                          uint64_t seed, void* stream, dpf_ctx** out);

/*
 * The Gaussian approximation of the mixture prior of x_t (Section 4.2, Table 2) in a
 * context of dpf_create_std: on != 0 draws x_t from the Gaussian with the mixture's mean
 * sum_j qbar_j m_j and covariance Q_x + sum_j qbar_j (m_j - mean)(m_j - mean)^T
 * (m_j = E[x_t | x_{t-1}, z_j]), as mean + chol(covariance) e with the same normals e;
 * everything else is unchanged (the component draw is then not used). A model whose x
 * transition is free of z is not affected. DPF_E_INVALID for other contexts.
 */
dpf_status dpf_set_gaussian_approx(dpf_ctx* ctx, int32_t on);

/* Inner diagnostics of the newest materialised state (the state of step t-1 after
 * step t, see dpf_read): each group's inner effective sample size
 * (sum_j W_j)^2 / sum_j W_j^2 with W = exp(lq), in [1, M]; their minimum and mean
 * over the N groups (host doubles). Synchronises the stream. */
dpf_status dpf_diag_inner(dpf_ctx* ctx, double* ess_min, double* ess_mean);

/*
 * Read an internal device array into host memory (tests and checkpoints).
 * `which` names the array; `bytes` must equal its size exactly:
 *   "lw" (N), "lwhat" (N*L), "xbb" (N*L*d1, [n][m][c]), "anc" (N int32),
 *   "sel" (N int32), "wout" (N, the outer weights fed to the resampler),
 *   "xm" (d1*N, [c][n]) and "zm" (d2*N, [c][n]): each outer particle's part of
 *   the filtered mean of the last step before the outer weighting (the weighted
 *   sum over its look-ahead draws), in the internal x-first coordinates,
 *   "x" (N*d1, [n][c]), "z" (d2*N*M, [c][n][j]), "lq" (N*M) - x/z/lq are the
 *   newest materialised state, which is that of step t-1 after step t (the
 *   inner update of step t runs at the start of step t+1), and "sel" holds the
 *   draws that chose it; "bidx" (N*M int32, the local-resampling ancestors of
 *   that inner update; only when debug recording is on);
 * "head": N x M x dout float, the learned proposal's head outputs of that
 *   inner update (with a proposal set and debug recording on);
 * "afeat" (N x (2 d1 + dy + 2 d2) float) and "ahead" (N x 2 d2 float): the
 *   outer-amortised proposal's group features and network outputs of that update;
 * "fallback" (N int32): 1 where that learned update fell back to the plain rule.
 * Element type: the context's precision (or int32). Synchronises the stream.
 */
dpf_status dpf_read(dpf_ctx* ctx, const char* which, void* host_dst, size_t bytes);

/*
 * Checkpoints. A state holds everything the next step reads: the newest
 * materialised particles (x, z, lq), the look-ahead products and the ancestors
 * of the last step, the last observation, the running evidence and the step
 * counter, with a header of the sizes. dpf_state_bytes gives its size;
 * dpf_get_state copies it into dst_device (device memory, caller-owned, at
 * least that many bytes); dpf_set_state loads one taken from a filter of the
 * same kind (LA-DPF, particle filter or DPF without look-ahead), model family
 * (the conditionally linear-Gaussian family, or which of the paper's models in
 * which decomposition), precision and sizes (d1, d2, dy, N, M, L; else
 * DPF_E_INVALID). The steps
 * after a restore equal those of the original filter when both have the same
 * seed. Both synchronise the stream.
 */
dpf_status dpf_state_bytes(dpf_ctx* ctx, size_t* bytes);
dpf_status dpf_get_state(dpf_ctx* ctx, void* dst_device, size_t bytes);
dpf_status dpf_set_state(dpf_ctx* ctx, const void* src_device, size_t bytes);

/* Record per-step debug arrays ("bidx") when enable != 0. */
dpf_status dpf_set_debug(dpf_ctx* ctx, int32_t enable);

/* Choose the tensor-core propagation z_new = A_zz z (3xTF32 on tcgen05, the
 * default) or the CUDA-core one, for variants that have both (FP32, d2 a
 * multiple of 8 with constants too large for a launch parameter, M = 128 or
 * 256; elsewhere the flag has no effect). Takes effect at the next step. */
dpf_status dpf_set_tensor_cores(dpf_ctx* ctx, int32_t enable);

/*
 * Time the main step kernel: when enable != 0, every later step brackets that
 * kernel with CUDA events on the context's stream; dpf_profile_read returns the
 * summed milliseconds and the number of timed launches, and resets them.
 */
dpf_status dpf_profile(dpf_ctx* ctx, int32_t enable);
dpf_status dpf_profile_read(dpf_ctx* ctx, double* kernel_ms, int64_t* launches);

/* Device bytes held by the context. */
dpf_status dpf_memory(dpf_ctx* ctx, size_t* bytes);

/* Free everything the context owns (NULL is a no-op). */
void dpf_destroy(dpf_ctx* ctx);

/*
 * Batched form: F independent filters stepped together (the many-filter
 * workload; each filter may have its own model, x/z split d1, N and M, but all
 * share d, dy, precision and L). Filter f uses seeds[f] (it reproduces a
 * single filter created with that seed). The filters of one compiled
 * (precision, d1, d2, dy) variant and inner-particles-per-lane class share one
 * persistent launch of the step kernel (or one launch each, where
 * dpf_batch_autotune finds that faster; always one each, on the batch's stream, for
 * the (8, 56, 8) variant, whose step reads its model from a shared constant
 * bank); the outer stages of the filters run concurrently. Each M must be at most 256 with M, L and L*d1 rows of whole
 * 16-byte units. models, d1, N, M, seeds: host arrays of F entries.
 */
typedef struct dpf_batch dpf_batch;
dpf_status dpf_batch_create(const dpf_model_desc* const* models, const int32_t* d1,
                            const int64_t* N, const int32_t* M, int32_t L, const uint64_t* seeds,
                            int32_t F, void* stream, dpf_batch** out);

/* One step of every filter: y_dev is device memory, F x dy (filter-major) of the
 * batch's precision; means_dev (F x d doubles) and logz_dev (F doubles, the
 * running log-evidence) are device outputs or NULL. Stream-ordered. */
dpf_status dpf_batch_step(dpf_batch* b, const void* y_dev, double* means_dev, double* logz_dev);

/* T steps from device observations ys_dev (T x F x dy); means_dev (T x F x d) and
 * logz_dev (T x F) are device outputs or NULL. With use_graph != 0 the whole run
 * is captured into one CUDA graph and launched once. Synchronises. */
dpf_status dpf_batch_run(dpf_batch* b, const void* ys_dev, int64_t T, double* means_dev,
                         double* logz_dev, int32_t use_graph);

/* Time the launch-shape candidates of every class on the live state (reps
 * launches each, without advancing the filters) and keep the fastest; a JSON
 * report of the choices is written to report (report_bytes, may be NULL). The
 * candidates are two inner-particles-per-lane counts, each as one launch for the
 * class (each filter's model constants staged in shared memory) or, for a class
 * of several filters, one launch a filter (its constants a launch parameter); the
 * results are the same under every choice.
 * DPF_E_INVALID before the first step: that step has no inner update, so its
 * launches would not time the steady-state kernel. */
dpf_status dpf_batch_autotune(dpf_batch* b, int32_t reps, char* report, size_t report_bytes);

/* Set the schedule of every class of several filters by hand, at the classes'
 * current inner-particles-per-lane: split != 0 one launch a filter, 0 one launch
 * a class (the schedule until dpf_batch_autotune chooses). The results are the
 * same under both; only the time differs. */
dpf_status dpf_batch_set_split(dpf_batch* b, int32_t split);

/* Borrow filter f's context (for dpf_read, dpf_diag); owned by the batch. */
dpf_status dpf_batch_filter(dpf_batch* b, int32_t f, dpf_ctx** out);

/* Wait for the batch and report latched device-side errors of any filter. */
dpf_status dpf_batch_sync(dpf_batch* b);

/* Time the batched step kernels with CUDA events (as dpf_profile). */
dpf_status dpf_batch_profile(dpf_batch* b, int32_t enable);
dpf_status dpf_batch_profile_read(dpf_batch* b, double* kernel_ms, int64_t* launches);

void dpf_batch_destroy(dpf_batch* b);

/*
 * ---- Learned inner proposal ----
 * Not in the paper: a learned replacement of the prior proposal of the inner
 * particles (Fig. 4, step 4; the r-tilde weight of eq. qbar):
 *   q_phi(z_t | f) = sum_c pi_c N(z_t; mu_c, diag sigma_c^2),
 *   f = (x_{t-1} of the ancestor, x_t, z_{t-1} of the resampled parent, y_t),
 * an MLP of three hidden ReLU layers (width `hidden`) with a head of
 * components (1 + 2 d2) outputs: logits, the means (component-major), then the
 * raw log standard deviations, clamped to [-7, 5] where used. Weights are FP32
 * master copies; every training product (forward and backward) runs on the tensor
 * cores with FP32 accumulation, on bfloat16 weights and activations by default, or
 * after dpf_proposal_set_bf16(p, 0) on FP32 operands as three TF32 products each
 * (about FP32 accuracy).
 *
 * Parameters (dpf_proposal_get/set_weights, host float arrays of num_params):
 *   W1 (hidden x din), b1, W2 (hidden x hidden), b2, W3, b3, W4 (dout x hidden), b4,
 * row-major, din = 2 d1 + d2 + dy <= 16, d2 <= 8, hidden a multiple of 16 up to
 * 256, 1..8 components, dout <= 128. The proposal is owned by the caller and
 * must outlive every filter that uses it.
 */
typedef struct dpf_proposal dpf_proposal;

dpf_status dpf_proposal_create(int32_t d1, int32_t d2, int32_t dy, int32_t hidden, int32_t components,
                               void* stream, dpf_proposal** out);
dpf_status dpf_proposal_num_params(const dpf_proposal* p, int64_t* n);
/* Load parameters (and reset Adam); n must equal num_params. Synchronises. */
dpf_status dpf_proposal_set_weights(dpf_proposal* p, const float* params, int64_t n);
dpf_status dpf_proposal_get_weights(const dpf_proposal* p, float* params, int64_t n);
/* Round the forward pass to bfloat16 (default, as the filter's tensor-core pass) or not. */
dpf_status dpf_proposal_set_bf16(dpf_proposal* p, int32_t enable);
/*
 * Weighted negative log-likelihood of n rows and its gradient: loss =
 * sum_b w_b (-log q(Z_b | F_b)) / sum_b w_b. F (n x din), Z (n x d2), w (n):
 * device float arrays; loss: host (may be NULL); grad_dev: device, num_params
 * floats in the parameter order, or NULL. Synchronises.
 */
dpf_status dpf_proposal_loss_grad(dpf_proposal* p, const float* F, const float* Z, const float* w, int64_t n,
                                  double* loss, float* grad_dev);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) with the given device gradient. Synchronises. */
dpf_status dpf_proposal_adam_step(dpf_proposal* p, const float* grad_dev, float lr);
/*
 * Train on n device rows (as dpf_proposal_loss_grad): `epochs` passes in
 * minibatches of `batch` rows, a fresh order each epoch (Fisher-Yates driven by
 * splitmix64 from `seed`), one Adam step per minibatch. losses: host, epochs
 * doubles (mean minibatch loss of each epoch), or NULL. Synchronises.
 */
dpf_status dpf_proposal_train(dpf_proposal* p, const float* F, const float* Z, const float* w, int64_t n,
                              int32_t batch, int32_t epochs, float lr, uint64_t seed, double* losses);
/*
 * The outer-amortised form: one network row per outer particle, whose head
 * gives a diagonal affine map (log s, c; 2 d2 outputs, log s clamped to
 * [-7, 5]) of that group's prior draws. Inputs (din = 2 d1 + dy + 2 d2): x_{t-1}
 * of the ancestor, x_t, y_t, and the mean m and per-coordinate variance v of the
 * group's prior means mu_j = A_zx x_{t-1} + A_zz z_{t-1}^(a, b_j); a particle's
 * prior draw zhat = mu_j + chol(Q_z) eps (PROP noise) becomes
 * z = m + c + s (zhat - m), weighted by log N(z; mu_j, Q_z) - log N(zhat; mu_j, Q_z)
 * + sum log s + log p(y_t | x_t, z). Qz: host, d2 x d2 (row-major), for the
 * training loss. Training rows (dpf_proposal_train, dpf_proposal_loss_grad):
 * F = the group features, Z = (z_t, mu_j, m) (3 d2 floats a row). d2 up to 64 and
 * din up to 160 (the mixture form: d2 up to 8, din up to 16).
 */
dpf_status dpf_proposal_create_amortised(int32_t d1, int32_t d2, int32_t dy, int32_t hidden, const double* Qz,
                                         void* stream, dpf_proposal** out);
/*
 * The centre k of the outer-amortised map z = k + c + s (zhat - k): 0 (default)
 * the group's mean prior mean m, 1 the particle's own prior mean mu_j (the map then
 * scales only the transition noise, which suits groups whose prior means spread
 * far wider than that noise). The weight keeps its form. Training rows then carry
 * the centre in their third block: Z = (z_t, mu_j, mu_j) (the recorded m replaced
 * by mu_j). DPF_E_INVALID for a mixture proposal or a value other than 0 or 1.
 */
dpf_status dpf_proposal_set_centre(dpf_proposal* p, int32_t per_particle);
/* The head outputs (n x dout floats, device) of n device feature rows by the
 * tensor-core forward pass the filter step uses at d = 4 (din <= 16, dout <= 32,
 * hidden 256; DPF_E_UNSUPPORTED otherwise). Synchronises. */
dpf_status dpf_proposal_forward(dpf_proposal* p, const float* F, int64_t n, float* out);
void dpf_proposal_destroy(dpf_proposal* p);

/*
 * Use `p` as the inner proposal of ctx from the next step on (NULL: the prior
 * again). Needs an FP32 context with d1, d2, dy equal to the proposal's; the
 * look-ahead is unchanged. The mixture form: (d1, d2, dy) = (2, 2, 2), hidden
 * 256, 4 components and M in {32, 64, 128}; the inner update then draws
 * z_t^(i,j) ~ q_phi(. | f) (component by the one-draw local systematic rule,
 * Philox purpose 10 = LCOMP, the normal noise from the PROP stream) and weights
 * it by log r = log p(z_t | z_{t-1}, x_{t-1}) - log q_phi(z_t | f) + log p(y_t | x_t, z_t).
 * The outer-amortised form (see dpf_proposal_create_amortised): (2, 2, 2) with
 * hidden 256 and M in {32, 64, 128, 256}, or (8, 56, 8) with an x transition free
 * of z and M a multiple of 32 up to 256 (the network's four products then run on
 * the tensor cores over the N group rows, any hidden width a multiple of 16).
 * DPF_E_UNSUPPORTED for other shapes.
 */
dpf_status dpf_set_proposal(dpf_ctx* ctx, dpf_proposal* p);

/*
 * Per-group fallback of the learned proposal to the plain inner update (the prior
 * proposal after local resampling, Fig. 4 step 4): after the learned update of a
 * step, a group whose inner effective sample size (sum_j W_j)^2 / sum_j W_j^2,
 * W = exp(lq) in FP32, is below frac * M (or has no finite weight) redoes its
 * inner update by the plain rule, with the same keys as a filter without a
 * proposal. frac in [0, 1]; 0 turns the fallback off; 0.25 when never set.
 * dpf_read(ctx, "fallback", ...) gives the last step's flags (N int32, 1 = fell
 * back).
 */
dpf_status dpf_set_fallback(dpf_ctx* ctx, double frac);

/*
 * Training rows from the inner update the last dpf_step ran (it must have run
 * one, with debug recording on: dpf_set_debug(ctx, 1)): for every inner
 * particle of the outer particles i0 .. i0 + n_outer - 1, F = (x_{t-1} of the
 * ancestor, x_t, z_{t-1} of the parent, y_t), Z = z_t and w = exp(lq_t) / N
 * (the normalised inner weight times the equal outer weight after resampling).
 * F: n_outer M x din, Z: n_outer M x d2, w: n_outer M; device floats. Synchronises.
 */
dpf_status dpf_record_tuples(dpf_ctx* ctx, int64_t i0, int64_t n_outer, float* F, float* Z, float* w);
/* The same rows for the outer-amortised form: G (n_outer M x (2 d1 + dy + 2 d2)),
 * Z (n_outer M x 3 d2: z_t, mu_j, m), w (n_outer M). Compiled for (d1, d2, dy) =
 * (2, 2, 2) and (8, 56, 8), M a multiple of 32 up to 256. */
dpf_status dpf_record_tuples_amortised(dpf_ctx* ctx, int64_t i0, int64_t n_outer, float* G, float* Z, float* w);

/*
 * A check of the failure path of the bounded waits; the paper has no
 * counterpart. Runs (1) the global resampling's scan on 3 x 2048 unit weights
 * with tile 0 publishing nothing, so that the look-back waits of the other
 * tiles can never be satisfied, and (2) a step's outer stage (3 CTAs of one
 * cooperative launch) with CTA 0 never reaching the grid-wide barrier. In both
 * the waits give up after their bound (a few tenths of a second) and the device
 * stays usable; the call returns DPF_E_TIMEOUT when both waits ran out as they
 * should, and another status otherwise. Synchronises the stream.
 */
dpf_status dpf_check_bounded_wait(void* stream);

/*
 * A check of the allocation-failure path; the paper has no counterpart. Arms a
 * host-side countdown: of the device allocations that contexts, batches and
 * proposals make from now on (dpf_create, dpf_create_pf, dpf_create_std,
 * dpf_set_debug, dpf_batch_create, dpf_proposal_create ...), the n-th fails as
 * if the device had no memory left, and the countdown is then spent. The call
 * that owns it returns DPF_E_NOMEM and releases whatever it had allocated.
 * n = 0 disarms; n < 0: DPF_E_INVALID. Process-wide; not for concurrent use.
 */
dpf_status dpf_fail_allocation_after(int64_t n);

/*
 * ---- Automatic state decomposition (Section "Automatic State Decomposition",
 * Fig. hedge) ----
 * Online bandits over K candidate decompositions (arms). Host code; no device.
 * DPF_HEDGE: full information. Round t draws from p_i(t) proportional to
 *   exp(eta G_i(t-1)); dpf_bandit_update(b, r) then takes the whole reward
 *   vector r(t) (K values in [0, 1]) and adds it to G.
 * DPF_EXP3: one arm a round. The draw is from phat_j(t) = (1 - gamma) p_j(t) +
 *   gamma / K; dpf_bandit_update(b, &r) takes the tried arm's reward r in [0, 1]
 *   and adds r / phat_{i_t}(t) to that arm's G (the simulated reward vector is
 *   zero elsewhere). dpf_bandit_choose must precede each update.
 * dpf_bandit_choose draws i_t by the inverse CDF of that distribution at
 * u = (w + 1/2) 2^-32, w the first word of Philox4x32-10 at counter
 * (t, 0, 11 << 24, 0) with key (seed_lo, seed_hi). dpf_bandit_probs gives the
 * current distribution (p for Hedge, phat for Exp3). Rewards outside [0, 1]:
 * DPF_E_INVALID.
 */
typedef struct dpf_bandit dpf_bandit;
enum { DPF_HEDGE = 0, DPF_EXP3 = 1 };
dpf_status dpf_bandit_create(int32_t kind, int32_t K, double eta, double gamma, uint64_t seed, dpf_bandit** out);
dpf_status dpf_bandit_probs(const dpf_bandit* b, double* p);
dpf_status dpf_bandit_choose(dpf_bandit* b, int32_t* action);
dpf_status dpf_bandit_update(dpf_bandit* b, const double* rewards);
/* Reward of an arm (Section 4.3): r = alpha / (alpha + |y - yhat|^2) in (0, 1], with
 * yhat the arm's one-step-ahead prediction of y (dy values each, host). For a
 * linear-Gaussian model, yhat_t = H A m_{t-1} from the arm's filtered mean m_{t-1}. */
dpf_status dpf_bandit_reward(const double* y, const double* yhat, int32_t dy, double alpha, double* r);
void dpf_bandit_destroy(dpf_bandit* b);

/* Message of the last failed call on this thread ("" if none). */
const char* dpf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DPF_H */
