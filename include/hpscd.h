/*
 * hpscd.h — C ABI of the GB300 (sm_103a) implementation of the HPSCD column
 * sweep, Algorithm 1 of N. P. Bakas, "Algorithmic Solution for Systems of
 * Linear Equations, in O(mn) time" (arXiv 2104.12570).
 *
 * Problem (Sec. 2, Eq. System): given X (m×n) and y (m), find a (n) with
 * X·a ≈ y, for tall (least squares), wide (consistent, infinitely many
 * solutions) and square systems.  Algorithm 1 sweeps the columns j = 1..n in
 * order; for each it forms da = <X_j, e> / <X_j, X_j> (Eq. da2), applies the
 * rank-1 correction e <- e - X_j·da (Eq. ek1-ek) and updates a_j <- a_j + da,
 * sweep after sweep, until the residual meets a threshold (Sec. 2, "break if
 * under a certain threshold").
 *
 * Conventions shared by every entry point:
 *   - All pointers named X, y, a (and their batched forms) are DEVICE pointers
 *     unless the function name ends in _host.  The caller owns them; X and y
 *     are never written.  No call keeps a pointer after it returns.
 *   - Column-major X: element (i, j) at X[j*ld + i], ld >= m.
 *     Row-major X:    element (i, j) at X[i*ld + j], ld >= n.
 *   - The residual is e = y - X·a (Algorithm 1, the initialisation of e).
 *   - hist[s] = ||e_s||_2 / ||y||_2 after sweep s (hist[0] is the residual of
 *     the initial guess); when y = 0 the absolute norm ||e_s||_2 is used.  The
 *     norms are accumulated in float64 on the device.
 *   - Stopping rules, tested once per sweep after column n:
 *       HPSCD_STOP_REL_RES:    stop after sweep s >= 0 when hist[s] <= tol,
 *                              tested on the true residual: the residual the
 *                              sweeps update is rounded to float32 at every
 *                              step, so when it first meets tol one more pass
 *                              over X recomputes e = y - X·a for the float32
 *                              coefficients to be returned (compensated,
 *                              float64-grade accumulation) and hist[s] becomes
 *                              that value; the solve stops if it meets tol and
 *                              otherwise sweeps on from the recomputed e
 *                              (hpscd_select tests the updated residual);
 *       HPSCD_STOP_REL_CHANGE: stop after sweep s >= 1 when
 *                              |hist[s-1] - hist[s]| < tol * hist[s-1]
 *                              (or hist[s-1] == 0);
 *       HPSCD_STOP_NONE:       run exactly max_sweeps sweeps.
 *   - A column with <X_j, X_j> = 0 is skipped (da = 0).
 *   - Every call is stream-ordered on the context's stream; the solve calls
 *     return after the result (a, hist, status) is complete.
 *   - Functions return an hpscd_status; nothing else crosses the ABI.  On
 *     HPSCD_ERR_NOT_CONVERGED and HPSCD_ERR_NONFINITE the outputs still hold
 *     the last iterate and its history.
 */
#ifndef HPSCD_H
#define HPSCD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HPSCD_OK = 0,
  HPSCD_ERR_INVALID_ARG = 1,   /* bad pointer, size, stride, enum or option */
  HPSCD_ERR_NOT_CONVERGED = 2, /* max_sweeps ran out before the stopping rule held */
  HPSCD_ERR_NONFINITE = 3,     /* a residual norm became NaN or Inf */
  HPSCD_ERR_TIMEOUT = 4,       /* a bounded device-side wait gave up */
  HPSCD_ERR_CUDA = 5,          /* a CUDA runtime call failed */
  HPSCD_ERR_UNSUPPORTED = 6,   /* shape/layout/dtype combination not provided */
  HPSCD_ERR_NO_MEMORY = 7      /* workspace allocation failed or is too small */
} hpscd_status;

/* Storage type of X.  Every type is widened exactly to float32 when read; the
 * arithmetic is the same for all three (float32 products and sums, float64
 * where stated). */
typedef enum { HPSCD_F32 = 0, HPSCD_BF16 = 1, HPSCD_F16 = 2 } hpscd_dtype;
typedef enum { HPSCD_COL_MAJOR = 0, HPSCD_ROW_MAJOR = 1 } hpscd_layout;
typedef enum {
  HPSCD_STOP_REL_RES = 0,
  HPSCD_STOP_REL_CHANGE = 1,
  HPSCD_STOP_NONE = 2
} hpscd_stop_rule;

/* Options of one solve.  Zero-initialise, then set the fields you need. */
typedef struct {
  double tol;            /* threshold of the stopping rule (>= 0) */
  int64_t max_sweeps;    /* N of Algorithm 1 (>= 0) */
  int32_t stop_rule;     /* hpscd_stop_rule */
  int32_t refresh_every; /* k > 0: every k-th residual pass recomputes the true
                            residual e = y - X·a with compensated (float64-grade)
                            accumulation instead of updating e; 0: only the
                            initial residual is recomputed */
  int32_t debug_flags;   /* 0 in normal use.  Bit 0 (HPSCD_DEBUG_STALL_BARRIER):
                            the first grid barrier waits for one arrival more
                            than there are CTAs, so its bounded wait runs out
                            and the solve returns HPSCD_ERR_TIMEOUT; it tests
                            the timeout path without faulting or hanging */
  int32_t reserved[5];   /* must be zero */
} hpscd_opts;

#define HPSCD_DEBUG_STALL_BARRIER 1
/* Bit 1: form G = X^T X with the CUDA-core kernel even where the tensor-core
 * (tcgen05) kernel applies (cross-checking the two). */
#define HPSCD_DEBUG_SIMT_GRAM 2
/* Bit 2: keep the residual e in HBM even where the tall sweep would keep the
 * rows of each CTA in shared memory (measuring the difference). */
#define HPSCD_DEBUG_E_IN_HBM 4

/* Timings of the last solve on a context, from CUDA events on its stream. */
typedef struct {
  float setup_ms;        /* <X_j,X_j> and Gram set-up kernels */
  float sweep_ms;        /* the persistent sweep kernel */
  int64_t passes;        /* streaming passes over X made by the sweep kernel */
  int64_t x_bytes;       /* bytes of X (m·n·element size) */
  int32_t grid;          /* CTAs of the sweep kernel */
  int32_t kernel_launches; /* kernels launched by the solve */
} hpscd_timing;

/* Result of one solve of a batch (hpscd_batch_results) or of an asynchronous
 * solve (hpscd_solve_async). */
typedef struct {
  int64_t sweeps;      /* sweeps made */
  double rel_res;      /* hist[sweeps] */
  int32_t status;      /* hpscd_status of the solve */
  int32_t passes;      /* streaming passes over its X */
} hpscd_sys_result;

typedef struct hpscd_ctx hpscd_ctx;

/* Create a context bound to CUDA device `device` and stream `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The context owns a
 * device workspace that grows on demand (cudaMalloc) unless the caller installs
 * one with hpscd_set_workspace.  Errors: INVALID_ARG, CUDA. */
int hpscd_create(hpscd_ctx** out, int device, void* stream);

/* Release the context and any workspace it allocated.  NULL is accepted.
 * Batches and networks made on the context keep it: destroyed while any of
 * them is alive, the context is only marked closed (no further calls on it)
 * and is freed when the last of them is destroyed. */
int hpscd_destroy(hpscd_ctx* ctx);

/* Rebind the context to another stream of the same device. */
int hpscd_set_stream(hpscd_ctx* ctx, void* stream);

/* Limit (seconds, > 0) of every device-side spin wait (grid barrier, copy
 * completion).  When it runs out the kernel stops, the call returns
 * HPSCD_ERR_TIMEOUT and the context stays usable.  Default 5 s. */
int hpscd_set_timeout(hpscd_ctx* ctx, double seconds);

/* Device workspace (bytes) a solve of this shape needs. */
int hpscd_workspace_size(hpscd_ctx* ctx, int dtype, int layout, int64_t m, int64_t n,
                         const hpscd_opts* opts, size_t* bytes);

/* Install caller-owned device memory as the workspace (256-byte aligned).  The
 * context never frees it; solves that need more return HPSCD_ERR_NO_MEMORY.
 * ptr = NULL returns the context to allocating its own. */
int hpscd_set_workspace(hpscd_ctx* ctx, void* ptr, size_t bytes);

/*
 * Solve X·a ≈ y by sweeps of Algorithm 1 (Sec. 2) on the GPU.
 *   X      device, dtype HPSCD_F32, HPSCD_BF16 or HPSCD_F16, layout/ld as above;
 *          every shape is taken (m, n >= 0), by one of three sweeps:
 *            column-major, n <= 512: the persistent tall sweep (tall and
 *              square systems; TMA tiles when X is 16-byte aligned and ld·size
 *              a multiple of 16, plain loads otherwise);
 *            column-major, n > 512: the persistent panel sweep (the columns in
 *              panels of 512 in the paper's order; X is read twice per sweep);
 *            row-major, m <= 4096: one thread-block cluster walks the column
 *              chain (wide systems); 16-bit X is first widened to a float32
 *              copy in the workspace (m·n·4 bytes, values exact);
 *            row-major, m > 4096: X is first transposed to a column-major
 *              copy in the workspace (n·m bytes of its own type), then as
 *              column-major.
 *          The copies are made once per call, as part of the set-up.
 *   y      device float[m].
 *   a      device float[n]; in: the initial guess when a_is_guess != 0
 *          (Algorithm 2's "or initial guess"), ignored otherwise (0_n);
 *          out: the coefficients after the last sweep.
 *   hist   HOST double[max_sweeps + 1] or NULL; entries past the last sweep
 *          are left untouched.
 *   sweeps_done, final_rel_res: HOST, may be NULL.
 * Returns OK when the stopping rule held, NOT_CONVERGED, NONFINITE, TIMEOUT,
 * INVALID_ARG, UNSUPPORTED, NO_MEMORY or CUDA.
 */
int hpscd_solve(hpscd_ctx* ctx, const void* X, int dtype, int layout, int64_t m, int64_t n,
                int64_t ld, const float* y, float* a, int a_is_guess, const hpscd_opts* opts,
                double* hist, int64_t* sweeps_done, double* final_rel_res);

/*
 * Algorithm 2 (HPSCDP, Sec. 7): the sweep of hpscd_solve with the columns taken
 * in blocks of thr consecutive columns (the last block holds the n mod thr
 * remaining ones); every column of a block takes its step
 * da_k = <X_k, e> / <X_k, X_k> against the SAME residual, then
 * e <- e - X_block·da_block.  thr = 1 is Algorithm 1, thr >= n a Jacobi
 * iteration; the paper finds convergence for thr around n/10, which is not
 * guaranteed in general.  Column-major X only (n <= 512); other arguments,
 * results and errors as hpscd_solve (INVALID_ARG for thr < 1).
 */
int hpscd_solve_blocks(hpscd_ctx* ctx, const void* X, int dtype, int64_t m, int64_t n, int64_t ld,
                       const float* y, float* a, int a_is_guess, int64_t thr,
                       const hpscd_opts* opts, double* hist, int64_t* sweeps_done,
                       double* final_rel_res);

/*
 * Algorithm 3 (HPSCDF, Sec. 8): greedy feature selection.  From a = 0, e = y,
 * each step forms da = (X^T e) ⊘ diag(X^T X) for every column, takes the column
 * jhat of least error E_j = sum_i (e_i - X_ij·da_j)^2 (lowest j on ties), and
 * adds it: a_jhat <- a_jhat + da_jhat, e <- e - X_jhat·da_jhat.  One step costs
 * one streaming pass over X.  opts->max_sweeps is the number of steps F; the
 * stopping rules apply per step on hist (REL_CHANGE stops once the errors stop
 * decreasing, the paper's while-loop variant); refresh_every must be 0.
 *   sel        HOST int64[max_sweeps]: the column chosen at each step (a column
 *              may be chosen again; the selected set is the distinct entries).
 *   a          DEVICE float[n], out: the coefficients (0 for unselected columns).
 *   hist       HOST double[max_sweeps + 1] or NULL: ||e|| / ||y|| after each step.
 *   steps_done, final_rel_res: HOST, may be NULL.
 * Column-major X (m >= 1, 1 <= n <= 512).  Errors as hpscd_solve.
 */
int hpscd_select(hpscd_ctx* ctx, const void* X, int dtype, int64_t m, int64_t n, int64_t ld,
                 const float* y, float* a, const hpscd_opts* opts, int64_t* sel, double* hist,
                 int64_t* steps_done, double* final_rel_res);

/*
 * Algorithm 1 with the column of every step given (Sec. 2: instead of taking
 * j = 1..n in turn, a step may take a randomly chosen index j).  Step k of
 * sweep s (k = 0..n-1, s = 1..max_sweeps) applies the column step of Eq. da2 /
 * Eq. ek1-ek to column order[(s-1)·n + k]; an index may repeat within a sweep
 * and a column may be left out.  The caller draws the indices.
 *   order  HOST int32[opts->max_sweeps · n], every entry in [0, n): copied to
 *          the workspace before the launch; max_sweeps · n <= 2^28.
 * A sweep is the restated pass of hpscd_solve with the substitution run over
 * the steps (couplings G~[order_k][order_l], gathered) and the steps of each
 * column summed in step order.  Float32 column-major X, n <= 512; refresh_every
 * is honoured.  Other arguments, results and errors as hpscd_solve
 * (INVALID_ARG for an index outside [0, n), UNSUPPORTED for bfloat16 X).
 */
int hpscd_solve_order(hpscd_ctx* ctx, const void* X, int dtype, int64_t m, int64_t n, int64_t ld,
                      const float* y, float* a, int a_is_guess, const int32_t* order,
                      const hpscd_opts* opts, double* hist, int64_t* sweeps_done,
                      double* final_rel_res);

/*
 * Asynchronous form of hpscd_solve for column-major X (m >= 1, 1 <= n <= 512):
 * enqueues the whole solve (set-up and sweep kernels) on the context's stream
 * and returns without waiting, so that consecutive solves run back to back.
 *   hist   DEVICE double[opts->max_sweeps + 1] or NULL: residual history.
 *   res    DEVICE hpscd_sys_result, written when the solve has
 *          finished: sweeps, rel_res, status (the hpscd_status hpscd_solve
 *          would return), passes.
 * X, y, a, hist and res must stay valid until the stream has passed the solve;
 * solves on one context share its workspace and run in stream order.  The
 * return value reports only argument and launch errors.  CUDA-event timings of
 * the most recent asynchronous calls: hpscd_async_timings.
 */
int hpscd_solve_async(hpscd_ctx* ctx, const void* X, int dtype, int64_t m, int64_t n, int64_t ld,
                      const float* y, float* a, int a_is_guess, const hpscd_opts* opts,
                      double* hist, hpscd_sys_result* res);

/* Waits for the context's stream, then writes the timings of the last `count`
 * asynchronous solves (oldest first; 1 <= count <= 64 and <= the number of
 * such calls made) to HOST out[count].  passes is -1 (it is in each call's
 * result). */
int hpscd_async_timings(hpscd_ctx* ctx, int64_t count, hpscd_timing* out);

/*
 * Algorithm 3 followed by the feature-removal loop of Sec. 8: after the F =
 * opts->max_sweeps selection steps of hpscd_select, at most swap_rounds swap
 * steps.  A swap step drops a selected column k (a_k != 0) and adds an
 * unselected column j refitted on the residual without k
 * (a_j = <X_j, e + X_k·a_k> / <X_j, X_j>, Eq. da2), choosing the pair of least
 * resulting error (lowest k, then j, on ties), and is made only if that error
 * is below the current one; the loop ends at the first step that finds none.
 * Each swap step costs one streaming pass over X (the couplings come from G).
 * If a stopping rule ends the selection before F steps, no swap is tried.
 *   sel    HOST int64[max_sweeps]: as hpscd_select.
 *   swaps  HOST int64[2·swap_rounds]: (k, j) of each swap made, -1 after.
 *   hist   HOST double[max_sweeps + swap_rounds + 1] or NULL: ||e||/||y|| after
 *          each selection step, then after each swap.
 *   steps_done: selection steps + swaps made.
 * Column-major X (m >= 1, 1 <= n <= 512); 0 <= swap_rounds <= 2^20.  Errors as
 * hpscd_select.
 */
int hpscd_select_swap(hpscd_ctx* ctx, const void* X, int dtype, int64_t m, int64_t n, int64_t ld,
                      const float* y, float* a, const hpscd_opts* opts, int64_t swap_rounds,
                      int64_t* sel, int64_t* swaps, double* hist, int64_t* steps_done,
                      double* final_rel_res);

/* Same as hpscd_solve but X, y and a are HOST pointers: the call copies X and y
 * to the device workspace, solves, and copies a back (an end-to-end call). */
int hpscd_solve_host(hpscd_ctx* ctx, const void* X, int dtype, int layout, int64_t m,
                     int64_t n, int64_t ld, const float* y, float* a, int a_is_guess,
                     const hpscd_opts* opts, double* hist, int64_t* sweeps_done,
                     double* final_rel_res);

/*
 * The Gram matrix G = X^T X of a column-major X (m×n, ld), the set-up of the
 * sweep: G_jj = <X_j, X_j> are the denominators of the column step (Eq. da2)
 * and G_jl (l < j) the couplings that Eq. ek1-ek introduces inside a sweep.
 * G: device float[n × ldG], row-major, both triangles written; ldG >= n.
 * Tensor cores (tcgen05) when X is TMA-aligned (16-byte base, ld·elem a
 * multiple of 16) and n <= 512 (bfloat16) or n <= 256 (float32; a two-term
 * tf32 split keeps float32-grade products); CUDA cores otherwise or with
 * flags = HPSCD_DEBUG_SIMT_GRAM.  Accumulation is float32 within a row block
 * and float64 across blocks.  Synchronous; timing in hpscd_last_timing.
 */
int hpscd_gram(hpscd_ctx* ctx, const void* X, int dtype, int64_t m, int64_t n, int64_t ld,
               float* G, int64_t ldG, int flags);

/* Timings of the last solve on this context. */
int hpscd_last_timing(hpscd_ctx* ctx, hpscd_timing* out);

/* Device-side phase trace of the persistent sweep (tracing; off by default).
 * max_passes > 0 enables it for the next solves (device memory is allocated
 * here, not in the solve); 0 disables it.  After a solve, hpscd_get_trace
 * copies to the host, for pass p < max_passes, six %globaltimer stamps (ns)
 * taken by CTA 0: [6p+0] pass start, [6p+1] end of its streaming, [6p+2] grid
 * barrier passed, [6p+3] partial sums reduced and g formed, [6p+5] forward
 * substitution done ([6p+4] is unused; unused fields stay 0); then, at
 * [6·max_passes + b], the time CTA b finished streaming in pass 1. */
int hpscd_set_trace(hpscd_ctx* ctx, int max_passes);
int hpscd_get_trace(hpscd_ctx* ctx, unsigned long long* out, int64_t words, int64_t* written);

/*
 * Allocation-free solve (no counterpart in the paper; an interface for callers
 * that cannot allocate device memory when they solve: cudaMalloc/cudaFree can
 * synchronize the device and stall other streams, and some callers run where a
 * framework's caching allocator or a fixed memory budget owns device memory).
 * Same arguments and stopping rules as hpscd_solve for a column-major X on the
 * CURRENT device, on `stream` (a cudaStream_t, NULL = default stream), with no
 * context: the call allocates nothing (no cudaMalloc, cudaFree or allocating
 * library routine).  X, y and a must be device (or managed) memory that the
 * current device addresses; anything else returns HPSCD_ERR_INVALID_ARG.
 * Its device scratch is one static 24 MiB array in the library, which every
 * GPU that loads the library holds until the process exits.
 * Limits: 1 <= m <= 1,048,576, 1 <= n <= 256, max_sweeps <= 4096 and
 * opts->debug_flags == 0; larger problems return HPSCD_ERR_UNSUPPORTED.
 * The set-up always forms G = X^T X on the CUDA cores (the tensor-core set-up
 * of hpscd_solve needs more partial storage than the array holds), so the
 * results agree with hpscd_solve's to float32 tolerance, not bit for bit.
 * The call is synchronous: it ends with a device-to-host copy of the result
 * into pageable memory and a stream synchronization, so it must not be issued
 * on a stream that is being captured.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current.
 * Every call shares the array and clears what must start at zero, so calls
 * that overlap on the GPU (other streams, other host threads) race and must be
 * serialized by the caller.  Device-side waits are bounded at 5 s.  hist,
 * sweeps_done and final_rel_res are HOST pointers (may be NULL).
 */
int hpscd_solve_noalloc(void* stream, const void* X, int dtype, int64_t m, int64_t n, int64_t ld,
                        const float* y, float* a, int a_is_guess, const hpscd_opts* opts,
                        double* hist, int64_t* sweeps_done, double* final_rel_res);

/* ---- batched solves (many independent systems, one persistent launch) ----
 *
 * The paper notes that solving many similar systems repeatedly is where the
 * method pays (Sec. 9); a batch sweeps every system of a list with Algorithm 1
 * (the same restated sweep and stopping rules as hpscd_solve) in ONE
 * persistent kernel launch, replayed from a CUDA graph captured once. */

/* One system of a batch.  All pointers are DEVICE pointers owned by the
 * caller; X column-major (element (i, j) at X[j*ld + i]). */
typedef struct {
  const void* X;       /* float32, m×n, ld >= max(m, 1) */
  const float* y;      /* float[m] */
  float* a;            /* float[n]: in: guess when a_is_guess != 0; out: coefficients */
  double* hist;        /* double[max_sweeps + 1] or NULL: residual history */
  int64_t m;           /* 0 <= m <= max rows of the batch (see hpscd_batch_create) */
  int64_t n;           /* 0 <= n <= 256 */
  int64_t ld;
  int32_t a_is_guess;
  int32_t reserved;    /* must be zero */
} hpscd_sys;

/* Result of one system of a batch: hpscd_sys_result (above). */

/* Launch shape of a batch.  cluster = CTAs that share one system (1, 2, 4 or
 * 8; each CTA owns a slice of its rows and of its residual); 0 = let the
 * library pick.  panel = the width of the column panels of a streaming pass,
 * as columns per warp: 0 = the narrowest that covers the system's columns
 * (4 for n <= 64, 8 for n <= 128, 16 above), 1 = twice that, 2 = 16 for every
 * system (wider panels: fewer row sums per panel, taller row panels).
 * hpscd_autotune_batch fills both by timing candidates. */
typedef struct {
  int32_t cluster;
  int32_t panel;
  int32_t reserved[6]; /* must be zero */
} hpscd_tuning;

typedef struct hpscd_batch hpscd_batch;

/*
 * Plan a batch of `count` systems (sys: HOST array of descriptors, copied;
 * the device buffers they point to must stay valid while the batch is used).
 * dtype must be HPSCD_F32.  Every system: 0 <= n <= 256 and m small enough
 * for its residual slice to stay in shared memory (m <= 16384 per CTA of a
 * cluster, i.e. m <= 16384·cluster); opts->refresh_every and debug_flags
 * must be 0.  The call allocates the batch's device workspace (descriptors,
 * queue order by decreasing m·n, per-cluster Gram slots, results) and captures
 * the launch sequence (queue reset, persistent kernel) in a CUDA graph on the
 * context's device.  Errors: INVALID_ARG, UNSUPPORTED, NO_MEMORY, CUDA.
 */
int hpscd_batch_create(hpscd_ctx* ctx, const hpscd_sys* sys, int64_t count, int dtype,
                       const hpscd_opts* opts, const hpscd_tuning* tuning, hpscd_batch** out);

/* Replay the batch's graph on the context's stream (asynchronous; the
 * systems' a and hist and the results are complete when the stream reaches
 * this point).  CUDA-event timing goes to hpscd_last_timing (sweep_ms). */
int hpscd_batch_launch(hpscd_batch* b);

/* Wait for the last launch and copy the per-system results to the HOST array
 * out[count].  Returns OK, or the first non-OK status among the systems. */
int hpscd_batch_results(hpscd_batch* b, hpscd_sys_result* out);

/* The tuning the batch was planned with. */
int hpscd_batch_tuning(hpscd_batch* b, hpscd_tuning* out);

/* Release the batch (waits for its last launch) and its hold on the warm-start
 * network and the context.  NULL is accepted. */
int hpscd_batch_destroy(hpscd_batch* b);

/*
 * Autotuner: plans the batch with each candidate (cluster 1, 2, 4, 8) × (panel
 * 0, 1, 2) that fits, times with CUDA events a launch of `trial_sweeps` sweeps
 * of every system and one of none (stop rule NONE; the systems' a and hist are
 * written as by a solve), and returns in *out the candidate whose sweeps take
 * least time (the difference; the set-up is paid once per solve).
 * ms_per_candidate: HOST double[12] or NULL, that sweep time of candidate
 * (cluster index c, panel p) at [3·c + p]; a candidate that does not fit reads
 * as a negative number.
 */
int hpscd_autotune_batch(hpscd_ctx* ctx, const hpscd_sys* sys, int64_t count, int dtype,
                         int64_t trial_sweeps, hpscd_tuning* out, double* ms_per_candidate);

/* ---- learned warm start (an initial guess, as Algorithm 2 allows, for
 * families of similar systems) ----
 *
 * A 3-layer MLP maps the features phi = [theta_1..16, n/256, log(m)/log(16384)]
 * of a system of a parametric family to a predicted a (256 outputs, of which
 * the first n are used): Linear(18, 256), ReLU, Linear(256, 256), ReLU,
 * Linear(256, 256).  Matrix operands are bfloat16 (weights and activations),
 * accumulation float32 on the tensor cores; master weights and Adam moments are
 * float32.  It is trained on solutions the sweep itself produces. */
typedef struct hpscd_mlp hpscd_mlp;

/* Create an MLP on the context's device for batches of up to max_batch rows.
 * Parameters start at zero: set them with hpscd_mlp_set_params.
 * Errors: INVALID_ARG, UNSUPPORTED (no tensor-map support), NO_MEMORY, CUDA. */
int hpscd_mlp_create(hpscd_ctx* ctx, int64_t max_batch, hpscd_mlp** out);
/* A network that batches start from (hpscd_batch_set_warm_start) is freed
 * when the last such batch lets go of it; until then only no further calls. */
int hpscd_mlp_destroy(hpscd_mlp* mlp);

/* Number of float32 parameters: W1 [256][18], b1 [256], W2 [256][256], b2,
 * W3 [256][256], b3, in this order, row-major (W[out][in]). */
int64_t hpscd_mlp_param_count(void);

/* Copy all parameters from / to a HOST float array of hpscd_mlp_param_count()
 * entries.  set_params also resets the Adam moments and step count. */
int hpscd_mlp_set_params(hpscd_mlp* mlp, const float* host_params);
int hpscd_mlp_get_params(hpscd_mlp* mlp, float* host_params);

/* Predictions out[b][0..255] (DEVICE float[B][256]) for theta (DEVICE
 * float[B][16]) and the HOST int64 arrays m[B], n[B] (0 <= n <= 256). */
int hpscd_mlp_predict(hpscd_mlp* mlp, const float* theta, const int64_t* m, const int64_t* n,
                      int64_t B, float* out);

/* Loss L = mean over b < B, j < n_b of (out[b][j] - target[b][j])^2 (target:
 * DEVICE float[B][256]) and its gradient with respect to every parameter,
 * copied to the HOST array host_grads (layout of the parameters); no update. */
int hpscd_mlp_gradients(hpscd_mlp* mlp, const float* theta, const int64_t* m, const int64_t* n,
                        const float* target, int64_t B, double* loss, float* host_grads);

/* One Adam step (Kingma and Ba 2015: learning rate lr, beta1, beta2, eps, bias
 * correction) on the loss of hpscd_mlp_gradients; *loss (HOST, may be NULL)
 * receives the loss before the step.  Synchronous. */
int hpscd_mlp_train_step(hpscd_mlp* mlp, const float* theta, const int64_t* m, const int64_t* n,
                         const float* target, int64_t B, float lr, float beta1, float beta2,
                         float eps, double* loss);

/* Make every launch of the batch start each system from the MLP's prediction:
 * the batch's graph is re-captured as [MLP forward on theta (DEVICE
 * float[count][16], row i = system i) -> a_i of each system -> the sweep].
 * mlp = NULL restores the descriptors' own a_is_guess.  The MLP and theta must
 * stay valid while the batch is launched. */
int hpscd_batch_set_warm_start(hpscd_batch* b, hpscd_mlp* mlp, const float* theta);

/* Static description of a status code. */
const char* hpscd_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* HPSCD_H */
