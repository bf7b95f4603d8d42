/*
 * odmd.h -- C ABI of the online dynamic mode decomposition (DMD) library for GB300.
 *
 * The library keeps a DMD model of a snapshot stream u^0, u^1, ... on one GPU and
 * updates it with one rank-1 step per snapshot, as in Suh, Chung, Bremer, Choi,
 * "Accelerating Flow Simulations using Online Dynamic Mode Decomposition" (NeurIPS
 * 2023 ML4PS workshop), Section 2.3:
 *
 *   U^- = [u^0 .. u^{m-1}] ~ L S R^T  (truncated SVD, rank r <= r_max)
 *   U^+ = [u^1 .. u^m]
 *   A~_r = L^T U^+ R S^{-1} = V Lambda V^{-1},  Phi = L V
 *   u(t) = Phi Lambda^t Phi^+ u(0)     (t in steps, counted from u^0)
 *
 * and exposes the credibility test of Section 2.2 as a relative L2 distance between a
 * prediction and a full-order-model (FOM) snapshot.  The update is Brand's rank-1
 * append (the method Section 2.3 adopts), kept in product form L = L0 Q: the tall
 * basis L0 (N x r0) only gains columns, the small r0 x r factor Q absorbs the
 * rotations, and L0 is compacted to L0 Q when r0 reaches r_max + slack.
 *
 * Conventions for every call
 * --------------------------
 * - Every function returns an odmd_status and never aborts.  ODMD_OK is 0.
 * - "device" pointers are CUDA global-memory addresses of the GPU the handle was
 *   created on; "host" pointers are ordinary CPU memory.  The caller owns all of them.
 * - Work is enqueued on the handle's stream (a cudaStream_t passed as void*; NULL is
 *   the legacy default stream).  Calls that return numbers to the host (check, get_*,
 *   sync) synchronise that stream; the others are asynchronous.  A device-side error
 *   (non-finite input, a solver that did not converge) is recorded on the device and
 *   reported by the next synchronising call.
 * - A handle is not thread-safe; different handles may be used concurrently.
 * - Snapshot element type: double for ODMD_FP64, float for ODMD_FP32.
 *   Snapshots are contiguous vectors of n elements.
 */
#ifndef ODMD_H
#define ODMD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct odmd_instance* odmd_t;

typedef enum {
  ODMD_OK = 0,
  ODMD_ERR_ARG = 1,      /* bad argument (null pointer, size out of range, misalignment) */
  ODMD_ERR_STATE = 2,    /* call not valid in the current state (e.g. predict before a model exists) */
  ODMD_ERR_NOMEM = 3,    /* workspace too small, or a host allocation failed */
  ODMD_ERR_CUDA = 4,     /* a CUDA runtime call failed; see odmd_last_error */
  ODMD_ERR_NUMERIC = 5,  /* non-finite input or result, or an ill-conditioned eigenbasis */
  ODMD_ERR_TIMEOUT = 6   /* a bounded device-side wait ran out */
} odmd_status;

/* Storage of the tall basis L0 (the arithmetic of the tall passes is always
 * compensated: products are formed exactly and summed in a two-float accumulator).
 *   ODMD_FP64: basis as an unevaluated sum of two floats (hi + lo, 48-bit significand),
 *              snapshots and outputs double.
 *   ODMD_FP32: basis float, snapshots and outputs float.
 *   ODMD_BF16: reserved; rejected with ODMD_ERR_ARG (a bfloat16 basis cannot stay
 *              orthonormal to the accuracy the rank-1 update assumes).
 * In every mode the core SVD and the operator update of an update are FP64; the eigensolve
 * and the modal coefficients of predictions are double-float (48-bit significand). */
typedef enum { ODMD_FP64 = 0, ODMD_FP32 = 1, ODMD_BF16 = 2 } odmd_precision;

typedef struct {
  int64_t n;            /* state length N, 1 <= n <= 2^31 - 1 */
  int32_t r_max;        /* rank cap, 1 <= r_max <= 64 */
  int32_t slack;        /* extra basis columns before compaction, 0 <= slack <= 32
                           (0: the tall basis is rotated on every update at full rank) */
  double trunc_tol;     /* tau: a new direction enters iff rho > tau*max(sigma_1, ||c||);
                           singular values <= tau*sigma_1 are dropped.  1e-13 <= tau < 1 */
  double check_tol;     /* default tolerance of odmd_check (Sec. 3 uses 1e-5) */
  odmd_precision prec;  /* basis storage, see above */
  int32_t refine_every; /* refine orthogonality after every this many pairs (0: never);
                           see odmd_refine */
  uint32_t flags;       /* 0, or ODMD_CUDA_CORES and/or ODMD_NO_PIPELINE; other bits are rejected */
} odmd_config;

/* flags: keep multi-horizon rollouts and compactions on the CUDA cores.  By default a
 * prediction of 8 to 64 states, and the compaction of the product-form basis, run as exact
 * split products on the tensor cores when the basis has at most 64 columns (FP64 storage,
 * r_max + slack <= 63 for a compaction) or 96 (FP32 storage); this flag keeps the CUDA-core
 * path (the same values to the double-float rounding level). */
#define ODMD_CUDA_CORES 1u
/* flags: run every update to its end before the next one starts.  By default an update's
 * core SVD and operator update (Sec. 2.3: they do not feed the next projection, which needs
 * only the new basis column and the projection of the snapshot) run beside the next
 * update's pass over the basis, and complete before any other call on the handle reads the
 * model; the results are bitwise the same either way. */
#define ODMD_NO_PIPELINE 2u

/* Fill *cfg with the defaults for a stream of length n and rank cap r_max:
 * slack 16, trunc_tol 1e-10, check_tol 1e-5, ODMD_FP64, refine_every 0, flags 0. */
odmd_status odmd_config_default(odmd_config* cfg, int64_t n, int32_t r_max);

/* Device bytes the handle needs (the workspace passed to odmd_create), so that a caller
 * can admit instances against free HBM before allocating anything. */
odmd_status odmd_footprint(const odmd_config* cfg, size_t* device_bytes);

/* Create a handle.  workspace_dev: device memory of at least odmd_footprint() bytes,
 * 256-byte aligned, owned by the caller and not touched by anyone else until
 * odmd_destroy returns; the library allocates no device memory of its own.  The
 * workspace is initialised on `stream` (asynchronously).  *out receives the handle. */
odmd_status odmd_create(const odmd_config* cfg, void* workspace_dev, size_t bytes,
                        void* stream, odmd_t* out);

/* Append snapshot u^k (device, n elements of the snapshot type, any alignment).
 * The first call stores u^0; every later call adds the pair (u^{k-1}, u^k): U^- gains
 * u^{k-1}, U^+ gains u^k, and the model is updated by one rank-1 step (Sec. 2.3).
 * The snapshot is copied into the workspace on the stream, so the caller may reuse
 * its buffer once the stream has passed this call.  Unless ODMD_NO_PIPELINE is set, the
 * last part of the update (core SVD, operator update, compaction) is enqueued with the next
 * update, beside its pass over the basis, or by the next other call on the handle; the
 * model any call observes is the same either way. */
odmd_status odmd_update(odmd_t h, const void* x_dev);

/* Predict u(t_j) = Re(Phi Lambda^{t_j} Phi^+ u^0) for j < k (Sec. 2.3).  t_host: k step
 * counts from u^0 (host, any real value >= 0).  out_dev: device, column j at
 * out_dev + j*ld elements of the snapshot type, ld >= n.  Needs a model (two
 * snapshots with a nonzero first one); the eigendecomposition is recomputed lazily
 * after updates.  Asynchronous. */
odmd_status odmd_predict(odmd_t h, const double* t_host, int32_t k, void* out_dev, int64_t ld);

/* Credibility check (Sec. 2.2): rel_err = ||u(t) - x_fom|| / ||x_fom|| (0 if both are
 * zero, +inf if only x_fom is), pass = rel_err <= tol (tol <= 0 selects the handle's
 * check_tol).  x_fom_dev: device snapshot.  The prediction is never written to memory.
 * Synchronises the stream; both outputs are host pointers (either may be NULL). */
odmd_status odmd_check(odmd_t h, double t, const void* x_fom_dev, double tol,
                       double* rel_err, int32_t* pass);

/* One step of the hybrid FOM/ROM loop (Sec. 2.1, Fig. 1) for the step t = number of
 * snapshots received so far.  x_fom_dev: the FOM's state at step t (device, n elements of
 * the snapshot type).  If a model exists, the ROM predicts u(t) and the credibility test of
 * Sec. 2.2 compares it with x_fom (rel_err as in odmd_check; tol <= 0 selects check_tol);
 * a credible prediction is taken as the new state, otherwise the FOM state is.  The state
 * taken is written to state_out_dev (device, n elements, must not alias x_fom_dev) and
 * appended to the model as the next snapshot, so the pairs stay contiguous (an accepted
 * prediction updates the DMD as a FOM state would).  Before a model exists the FOM state is
 * taken.  *accepted (host, may be NULL): 1 if the prediction was taken; *rel_err (host, may
 * be NULL): the distance measured, +inf when no model existed.  Synchronises the stream
 * for the test; the update itself is asynchronous. */
odmd_status odmd_hybrid_step(odmd_t h, const void* x_fom_dev, double tol, void* state_out_dev,
                             int32_t* accepted, double* rel_err);

/* Append `count` snapshots read from host memory: snapshot k (n elements of the snapshot
 * type, double for ODMD_FP64 and float for ODMD_FP32) starts at element k*ld of host
 * (ld >= n).  Each is copied into one of two staging slots of the workspace on a copy
 * stream of the handle's own, and odmd_update runs on it once its copy has arrived; a slot
 * is refilled only after the update that read it, so with pinned host memory the copy of
 * snapshot k+1 overlaps the update of snapshot k.  Returns once the work is enqueued
 * (pageable host memory is copied before the call returns); a pinned buffer must stay
 * valid until the handle's stream has finished it (odmd_sync).  Errors: ODMD_ERR_ARG,
 * ODMD_ERR_CUDA, and those of odmd_update. */
odmd_status odmd_update_host(odmd_t h, const void* host, int64_t count, int64_t ld);

/* Many instances in one call (independent simulations, Sec. 2.1 per instance):
 * odmd_update_batch is odmd_update(hs[i], xs[i]) for i < count, and odmd_predict_batch is
 * odmd_predict(hs[i], ts[i], ks[i], outs[i], lds[i]).  Handles must be distinct within a
 * call; xs[i] is a device array of the handle's n elements in its snapshot format.
 * The update runs instances of the same storage format and compaction kind together: one
 * launch per step of the update (ingest, pass A, the five small-solve kernels, the
 * compaction) over all of them, each CTA doing what it does in its instance's own launch,
 * so every instance's result is bitwise that of odmd_update.  Such a group is split into S
 * sub-batches balanced by rows, each a CUDA graph on its own stream, so that the small solves
 * of one overlap the tall passes of another; S is picked by a tuner that times S = 1, 2, 4, 8
 * (as the group's size allows) on the first calls for the same set of handles (those calls
 * wait for their own step), then keeps the fastest.  The launches are ordered after each
 * handle's earlier work and before its later work on its stream.  Instances that cannot join
 * (their first snapshot, profiling on, row shards, another device) are updated one by one.
 * The group's plan (graphs and streams, no device memory) is kept until one of its handles
 * is destroyed or changes its row shards.  On a failure the call returns that status;
 * odmd_last_error(NULL) says which step or instance failed. */
odmd_status odmd_update_batch(odmd_t* hs, const void* const* xs, int32_t count);
odmd_status odmd_predict_batch(odmd_t* hs, const double* const* ts, const int32_t* ks, void* const* outs,
                               const int64_t* lds, int32_t count);

/* The sub-batch split S the tuner chose for the group of these handles, in this order: S >= 1
 * once chosen, 0 while it is still timing, -1 if no call has run this set as one group. */
odmd_status odmd_get_batch_split(odmd_t* hs, int32_t count, int32_t* split);

/* Orthogonality refinement (no counterpart in the paper: it keeps L^T L = I over long
 * streams, where rounding in every rank-1 update lets it drift, most of all with FP32
 * storage).  One pass over the basis forms C = L^T L; with C = R^T R (Cholesky) and
 * R diag(S) = U_s Sigma V_s^T the basis becomes L R^-1 U_s, orthonormal to working
 * accuracy, and S, the rows of the right factor and the reduced operator are rotated to
 * match, so the factorisation of the snapshots and the span of L are unchanged.  Runs
 * automatically after every refine_every-th snapshot pair when refine_every > 0 (which
 * also reserves its scratch in the workspace); otherwise this call returns
 * ODMD_ERR_STATE.  Asynchronous. */
odmd_status odmd_refine(odmd_t h);

/* Wait for the handle's stream and report any recorded device-side error. */
odmd_status odmd_sync(odmd_t h);

/* Current rank r (synchronises). */
odmd_status odmd_get_rank(odmd_t h, int32_t* r);

/* Singular values S (descending, host, up to cap of them) and the rank (synchronises). */
odmd_status odmd_get_singular_values(odmd_t h, double* s_host, int32_t cap, int32_t* r);

/* DMD eigenvalues Lambda (host re/im arrays, up to cap) and, if amp_host is not NULL,
 * each mode's amplitude |b_i| ||Phi e_i|| with b = Phi^+ u^0 (synchronises). */
odmd_status odmd_get_eigs(odmd_t h, double* re_host, double* im_host, double* amp_host,
                          int32_t cap, int32_t* r);

/* Write the orthonormal basis L = L0 Q (n x r, column-major, leading dimension ld >= n,
 * snapshot type) to out_dev and its rank to *r (synchronises to learn r first; out_dev
 * must hold r_max columns). */
odmd_status odmd_get_basis(odmd_t h, void* out_dev, int64_t ld, int32_t* r);

/* Number of snapshots received and number of compactions performed (host counters). */
odmd_status odmd_get_counts(odmd_t h, int64_t* snapshots, int64_t* compactions);

/* Kernel classes for odmd_profile_read. */
typedef enum {
  ODMD_K_PASS_A = 0,   /* tall projection/residual pass of an update */
  ODMD_K_SMALL = 1,    /* small solves of an update (5 kernels) */
  ODMD_K_PASS_B = 2,   /* tall append or compaction pass of an update */
  ODMD_K_EIG = 3,      /* eigensolve of the reduced operator */
  ODMD_K_COEF = 4,     /* modal coefficients of a rollout or check */
  ODMD_K_ROLLOUT = 5,  /* tall rollout pass (predict, basis export) */
  ODMD_K_CHECK = 6,    /* tall fused credibility-check pass */
  ODMD_K_FIRST = 7,    /* norm of the first snapshot */
  ODMD_K_REFINE = 8,   /* orthogonality refinement (Gram pass + 4 small kernels) */
  ODMD_K_GAP = 9,      /* two event records back to back inside a profiled update graph: the
                          overhead each bracketed group's time above includes */
  ODMD_K_COUNT = 10
} odmd_kernel_class;

/* Observability: when enabled (nonzero), every kernel group the handle enqueues is
 * bracketed by CUDA events on the handle's stream, and the time between them is
 * accumulated per class; enabling (or disabling) resets the accumulators.  This adds
 * two event records per group and nothing else. */
odmd_status odmd_profile_enable(odmd_t h, int32_t enable);

/* Read the accumulators (synchronises).  ms_total[c] and launches[c] for the first
 * `cap` classes (host arrays; either may be NULL): event time summed over the profiled
 * groups and the number of kernels launched since the handle was created.  mean_r0
 * (may be NULL) receives the mean number of basis columns r0 streamed by the profiled
 * pass-A launches. */
odmd_status odmd_profile_read(odmd_t h, double* ms_total, int64_t* launches, int32_t cap, double* mean_r0);

/* One step of the hybrid FOM/ROM loop with the paper's own credibility test (Sec. 2.2:
 * the residual of the FOM's discrete system at the predicted state).
 *
 * The step taken is t = number of snapshots received so far.  With a model, the library
 * predicts u(t) into state_out_dev and calls residual(user, t, state_out_dev, r_dev, b_dev,
 * stream): the caller's host function enqueues on `stream` (the handle's stream, a
 * cudaStream_t) the work that writes the right-hand side b of the FOM's step t into b_dev
 * and the residual r = b - A u of the predicted state into r_dev, and returns 0 (nonzero
 * reports a failure).  The library then forms ||r|| / ||b|| on the device (FP64 sums) and
 * accepts the prediction when it is <= tol (tol <= 0: the handle's check_tol).  Without a
 * model, or when the prediction is refused, it calls fom(user, t, state_out_dev, stream),
 * which enqueues the FOM's solve of step t into state_out_dev.  The state taken joins the
 * snapshot stream (odmd_update).  The callbacks keep whatever history their FOM needs:
 * before the call, state_out_dev holds nothing the library reads.
 *
 * state_out_dev, r_dev, b_dev: three distinct device buffers of n elements of the snapshot
 * type (double for ODMD_FP64, float for ODMD_FP32), owned by the caller.  accepted (1 if
 * the prediction was taken) and rel_res (the relative residual, +inf when no prediction
 * was made) are host outputs, either may be NULL.  Synchronises once per step with a
 * model.  Errors: ODMD_ERR_ARG (NULL or aliased pointers), ODMD_ERR_STATE (a callback
 * returned nonzero), ODMD_ERR_CUDA, ODMD_ERR_NUMERIC (non-finite residual). */
typedef int32_t (*odmd_residual_fn)(void* user, int64_t step, const void* u_dev, void* r_dev, void* b_dev,
                                    void* stream);
typedef int32_t (*odmd_fom_fn)(void* user, int64_t step, void* u_dev, void* stream);
odmd_status odmd_hybrid_step_residual(odmd_t h, odmd_residual_fn residual, odmd_fom_fn fom, void* user, double tol,
                                      void* state_out_dev, void* r_dev, void* b_dev, int32_t* accepted,
                                      double* rel_res);

/* The hybrid loop up to t_final with the convergence exit of Sec. 2.1:
 * steps t = (snapshots so far) .. t_final are taken with odmd_hybrid_step_residual (same
 * callbacks, buffers and tol).  Every check_every-th step, once a model exists, the DMD
 * eigenvalues of the modes that carry the field (amplitude >= 1e-6 of the largest) are
 * compared with those of the previous check; the paper does not define convergence, and
 * the reading taken is: conv_checks consecutive checks with the rank unchanged and every
 * such eigenvalue within conv_tol of the nearest one of the previous check.  Then the
 * remaining steps are skipped and u(t_final) is predicted into state_out_dev directly.
 * Otherwise state_out_dev ends holding the state taken at t_final.
 *
 * prev_dev: a fourth device buffer of n elements (caller's): on entry it must hold the
 * state taken at the step before the first one of the run; after every step the library
 * copies the state taken into it, so the callbacks of step t read u(t-1) there (state_out
 * holds the prediction of step t while they run).
 *
 * report (host, may be NULL): steps taken, FOM calls, accepted predictions, whether the
 * model converged, the step at which it did (-1 if not) and the steps skipped.  A check
 * whose eigensolve fails (no convergence, ill-conditioned eigenbasis) counts as not
 * converged.  Errors: those of odmd_hybrid_step_residual; ODMD_ERR_ARG for t_final before
 * the next step, check_every or conv_checks < 1, conv_tol <= 0. */
typedef struct {
  int64_t steps, fom_calls, accepted;
  int32_t converged, pad;
  int64_t converged_at, skipped;
} odmd_run_report;
odmd_status odmd_hybrid_run(odmd_t h, odmd_residual_fn residual, odmd_fom_fn fom, void* user, double tol,
                            int64_t t_final, int32_t check_every, int32_t conv_checks, double conv_tol,
                            void* state_out_dev, void* prev_dev, void* r_dev, void* b_dev, odmd_run_report* report);

/* Checkpoint / resume (the paper has no counterpart).
 *
 * odmd_checkpoint_size: bytes of a checkpoint of this handle (host memory).
 * odmd_save: synchronises, then writes the model's whole state into host_buf (bytes >=
 *   odmd_checkpoint_size): a header (magic, format version 2, n, r_max, precision, slack,
 *   snapshot count, indices of the committed buffers, region sizes, and an FNV-1a checksum
 *   over 8-byte little-endian words of the header with its checksum field zero and then of
 *   every region) followed by the raw device state -- control block, committed
 *   state buffers with the small scratch, rows 0..n-1 of the tall factor, both snapshot
 *   slots and the stored residual.  The host buffer is the caller's; nothing is kept.
 * odmd_load: restores such a checkpoint into a handle created with the same n, r_max,
 *   precision and slack (trunc_tol, check_tol and refine_every are the new handle's), on
 *   a device of the same kind.  Updates, predictions and checks then continue exactly as
 *   they would have in the saved handle.  Errors: ODMD_ERR_ARG for a NULL pointer, a
 *   short or truncated buffer, a foreign or corrupted checkpoint (bad magic, version or
 *   checksum; buffer indices other than 0 or 1, a negative snapshot count, or a control
 *   block that disagrees with the header, all refused before anything is copied to the
 *   device) or a different configuration; ODMD_ERR_CUDA. */
odmd_status odmd_checkpoint_size(odmd_t h, size_t* bytes);
odmd_status odmd_save(odmd_t h, void* host_buf, size_t bytes);
odmd_status odmd_load(odmd_t h, const void* host_buf, size_t bytes);

/* Row shards (Sec. 2.3: the O(N r) passes of an update are row-local, so the rows split
 * across GPUs and each pass ends in a reduction of a few values).  The paper has no
 * multi-GPU counterpart; this is the one-GPU form of a row-sharded run.
 *
 * The rows are cut into B row blocks, the same for every pass that ends in a reduction (the
 * projection/residual pass of an update, the credibility check, the norm of the first
 * snapshot): block b is rows [rows[b], rows[b+1]) with B and rows from odmd_get_row_blocks
 * (rows_host: cap >= B + 1 int64 on the host, may be NULL; block boundaries are multiples
 * of 64 rows).  Each block's partial sums are added in block order.
 *
 * odmd_set_row_shards: run every such pass as `shards` launches, shard g taking the
 * contiguous blocks [g B / shards, (g + 1) B / shards), each launch leaving its per-block
 * partials in the workspace, followed by one launch that adds all partials in block order
 * (the exchange a run on `shards` GPUs would make, an all-gather of the per-block partials).
 * The results are bitwise those of shards = 1 (the default), because every block's partial
 * and the order of the final sum are the same.  1 <= shards <= B, else ODMD_ERR_ARG.
 * Synchronises the stream; the captured update graphs are rebuilt on the next update. */
odmd_status odmd_set_row_shards(odmd_t h, int32_t shards);
odmd_status odmd_get_row_blocks(odmd_t h, int32_t* blocks, int64_t* rows_host, int32_t cap);

/* Release the handle (synchronises first).  The workspace is the caller's again. */
odmd_status odmd_destroy(odmd_t h);

/* Credibility check of a prediction the caller already holds, allocating nothing.
 * The paper has no counterpart: this is a convenience beside odmd_check for callers that
 * must not allocate device memory -- for example a callback inside a host solver's time
 * loop whose memory belongs to the solver's own pool allocator, a process under a hard
 * device-memory cap, or code that must avoid the device-wide synchronisation that
 * cudaMalloc/cudaFree can cause.  It needs no handle and no workspace.
 *
 *   rel_err = ||pred - x_fom|| / ||x_fom||  (0 if both are zero, +inf if only x_fom is),
 *   pass    = rel_err <= tol  (tol <= 0 selects 1e-5).
 *
 * pred_dev, x_fom_dev: device arrays of n doubles on the current device, read only.
 * n: 1 <= n <= 33,554,432; larger n is rejected with ODMD_ERR_ARG (the scratch is a fixed
 * 64 KiB device array inside the library, one partial-sum slot per 8192 elements).
 * stream: cudaStream_t as void* (NULL = legacy default stream); the call synchronises it.
 * rel_err, pass: host outputs (either may be NULL).  Sums are FP64.  Errors: ODMD_ERR_ARG,
 * ODMD_ERR_CUDA, ODMD_ERR_NUMERIC (non-finite input); the message is odmd_last_error(NULL).
 *
 * Every call synchronises its stream and copies the result to the host, so no call can be
 * captured into a CUDA graph.  The first call on each device loads the library's kernels
 * there (under lazy module loading) and looks up the scratch array's device address: make
 * one warm-up call at start-up, outside any section that must not allocate.  Every call in
 * the process shares the one array on a device: calls whose GPU work overlaps (different
 * streams or threads at the same time) race and may return wrong results. */
odmd_status odmd_check_noalloc(const double* pred_dev, const double* x_fom_dev, int64_t n, double tol,
                               void* stream, double* rel_err, int32_t* pass);

/* Message describing the last error on this handle (or the last global error if h is
 * NULL).  The string lives until the next call on the same handle. */
const char* odmd_last_error(odmd_t h);

/* ---------------------------------------------------------------- pairs (FOM-only updates)
 * Online DMD fed snapshot pairs (x, y = FOM(x)) that need not be contiguous: the hybrid
 * loop of Sec. 2 (Fig. 1) in the reading where only FOM steps update the model, so the
 * state a FOM step starts from may be an accepted DMD state rather than the previous
 * pair's y.  Sec. 2.3's matrices become X = [x_1 .. x_m] ~ L S R^T, Y = [y_1 .. y_m],
 * A~_r = L^T Y R S^{-1}; the handle keeps L and P = Y R (N x r each, double-float rows), S
 * and M = L^T P.  Snapshots, states and outputs are double, length n, contiguous, on the
 * device of the handle; FP64 accuracy only.  Errors are read with odmd_pairs_last_error.
 */
typedef struct odmd_pairs_instance* odmd_pairs_t;

/* Device bytes a pairs handle of length n and rank cap r_max (1..64) needs. */
odmd_status odmd_pairs_footprint(int64_t n, int32_t r_max, size_t* device_bytes);

/* Create a handle on a caller-owned workspace (256-byte aligned, at least
 * odmd_pairs_footprint bytes; the library allocates no device memory).  trunc_tol is tau
 * of odmd_config (a new direction enters iff rho > tau max(sigma_1, ||x||); singular values
 * <= tau sigma_1 are dropped), in [1e-13, 1).  stream: a cudaStream_t as void*. */
odmd_status odmd_pairs_create(int64_t n, int32_t r_max, double trunc_tol, void* workspace_dev, size_t bytes,
                              void* stream, odmd_pairs_t* out);

/* Append the pair (x, y): X gains x, Y gains y (asynchronous; a numerical failure of the
 * update is reported by the next synchronising call, and the model is then unchanged). */
odmd_status odmd_pairs_update(odmd_pairs_t h, const double* x_dev, const double* y_dev);

/* out[:, j] = L A~^{t_j} L^T u for k <= 64 integer horizons t_j in [0, 1e12] (steps after
 * the state u); column j at out + j*ld, ld >= n.  Synchronises the stream.
 * ODMD_ERR_STATE before the first pair with a nonzero x. */
odmd_status odmd_pairs_predict(odmd_pairs_t h, const double* u_dev, const double* t_host, int32_t k, double* out_dev,
                               int64_t ld);

/* Rank r and the min(r, cap) singular values of X, descending (synchronises). */
odmd_status odmd_pairs_get_singular_values(odmd_pairs_t h, double* s_host, int32_t cap, int32_t* r);

/* Step `step` of the hybrid loop of Sec. 2 (Fig. 1) in the FOM-only reading, with the
 * paper's residual test (Sec. 2.2).  On entry state_dev holds u^{k-1}; on return u^k.
 * With a model, next_dev receives the prediction L A~ L^T u^{k-1} and
 * residual(user, step, next_dev, r_dev, b_dev, stream) enqueues the FOM's residual
 * r = b - A u of it and its right-hand side b (state_dev still holds u^{k-1}); the
 * prediction is taken, without updating the model, when ||r|| / ||b|| <= tol (tol <= 0:
 * 1e-5, Sec. 3).  Otherwise next_dev receives u^{k-1}, fom(user, step, next_dev, stream)
 * enqueues the FOM's solve into it in place, and the pair (u^{k-1}, u^k) updates the model.
 * Four distinct device buffers of n doubles, owned by the caller; accepted and rel_res
 * (+inf without a prediction) are host outputs, either may be NULL.  Synchronises.
 * Errors: ODMD_ERR_ARG (NULL or aliased buffers), ODMD_ERR_STATE (a callback returned
 * nonzero), ODMD_ERR_NUMERIC (non-finite residual), ODMD_ERR_CUDA. */
odmd_status odmd_pairs_hybrid_step_residual(odmd_pairs_t h, odmd_residual_fn residual, odmd_fom_fn fom, void* user,
                                            double tol, int64_t step, double* state_dev, double* next_dev,
                                            double* r_dev, double* b_dev, int32_t* accepted, double* rel_res);

/* Pairs appended so far (host counter, no synchronisation). */
odmd_status odmd_pairs_get_count(odmd_pairs_t h, int64_t* pairs);

/* Message of the last failure on h (or of a call that had no handle when h is NULL). */
const char* odmd_pairs_last_error(odmd_pairs_t h);

/* Release the handle (synchronises first); the workspace is the caller's again. */
odmd_status odmd_pairs_destroy(odmd_pairs_t h);

/* ---------------------------------------------------------------- tensor-core self-test
 * The paper has no counterpart: a check of the hardware building block under the
 * split-precision tall x small products (bfloat16 tcgen05.mma into an FP32 accumulator in
 * tensor memory, canonical K-major shared-memory layout without swizzle).  One CTA forms
 * D = reps * A B with A 128 x 64 (row-major bfloat16 bits), B given as 64 rows of 64 (row
 * n holds column n of the 64 x 64 factor) and D 128 x 64 floats, row-major; all three and
 * the status word are device pointers owned by the caller.  1 <= reps <= 4096.
 * Synchronises the device.  Errors: ODMD_ERR_ARG, ODMD_ERR_CUDA, ODMD_ERR_TIMEOUT (the
 * product did not complete within the bounded wait; *status_dev is then nonzero). */
odmd_status odmd_tc_selftest(const void* a_dev, const void* b_dev, void* d_dev, int32_t* status_dev, int32_t reps);

#ifdef __cplusplus
}
#endif
#endif /* ODMD_H */
