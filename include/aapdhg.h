/*
 * aapdhg.h -- C ABI of the GB300 (sm_103a) AA-PDHG / FAA-PDHG LP solver.
 *
 * Method: arXiv 2508.08062.  The solver iterates the PDHG fixed-point map T
 * (Sec. 3, eq. pdhg / eq. new-fixed-point) with Anderson acceleration in the
 * regularised quasi-Newton form of Alg. 2 (AA-PDHG) or with the angle/length
 * filters of Alg. 3-6 (FAA-PDHG), a safeguard, and a projection back onto
 * X x Y.  Termination uses the relative KKT residual of the Remark on
 * termination conditions.
 *
 * LP form (Sec. 2.1, eq. LP-O):
 *     min c'x   s.t.  Gx >= h,  Ax = b,  l <= x <= u
 * K = [G; A] is passed as one CSR matrix with one sense byte per row
 * (AAPDHG_ROW_GE for a row of G, AAPDHG_ROW_EQ for a row of A), rows of
 * either kind in any order, and q = [h; b] in the same row order (eq.
 * lambda-case).  A "<=" row is passed negated as a ">=" row.
 *
 * Conventions of every entry point:
 *  - Plain C types only; no C++ exception crosses the boundary.
 *  - Host arrays passed in are copied; the caller keeps ownership.
 *  - Output pointers are caller-owned host buffers of the stated length.
 *  - Device memory of a handle is owned by the library and freed by
 *    aapdhg_destroy; it comes from the allocator installed with
 *    aapdhg_set_allocator (default cudaMalloc / cudaFree).
 *  - All device work of a handle is ordered on the handle's CUDA stream.
 *    A handle must not be used by two host threads at once.
 *  - Errors are sticky: after a call returns an error other than
 *    AAPDHG_NOT_CONVERGED, later calls on the handle return the same status
 *    until aapdhg_destroy.  aapdhg_last_error gives a message.
 */
#ifndef AAPDHG_H
#define AAPDHG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct aapdhg_s *aapdhg_t;

typedef enum {
    AAPDHG_OK = 0,
    AAPDHG_ERR_INVALID = 1,     /* bad argument or malformed CSR               */
    AAPDHG_ERR_OOM = 2,         /* device allocation failed                     */
    AAPDHG_ERR_CUDA = 3,        /* a CUDA runtime call failed                   */
    AAPDHG_ERR_NUMERIC = 4,     /* NaN/Inf in the iterate or the KKT residual   */
    AAPDHG_ERR_TIMEOUT = 5,     /* the run's time limit ran out (not sticky)    */
    AAPDHG_NOT_CONVERGED = 6    /* iteration cap reached with KKT > tol         */
} aapdhg_status;

enum { AAPDHG_ROW_EQ = 0, AAPDHG_ROW_GE = 1 };
enum { AAPDHG_FP64 = 0, AAPDHG_MIXED = 1 };     /* precision of iterates / SpMV   */
enum { AAPDHG_PDHG = 0, AAPDHG_AA = 1, AAPDHG_FAA = 2 };
enum { AAPDHG_MEM_HOST = 0, AAPDHG_MEM_DEVICE = 1 };
enum { AAPDHG_MAX_MEMORY = 32 };                /* largest m_A                    */

/* Device allocator used for every device buffer of handles created after the
 * call (process-wide).  alloc returns NULL on failure.  Passing NULL for both
 * restores cudaMalloc / cudaFree.  Always returns AAPDHG_OK.                  */
typedef void *(*aapdhg_alloc_fn)(size_t bytes, void *ctx);
typedef void (*aapdhg_free_fn)(void *ptr, void *ctx);
aapdhg_status aapdhg_set_allocator(aapdhg_alloc_fn alloc, aapdhg_free_fn free_fn, void *ctx);

/* Create a solver for the LP of eq. LP-O (Sec. 2.1).
 *   m, n        rows of K (m1 + m2 >= 0) and variables (n >= 1)
 *   nnz         entries of K, 0 <= nnz < 2^31
 *   row_ptr     int64[m + 1], row_ptr[0] = 0, non-decreasing, row_ptr[m] = nnz
 *   col_idx     int32[nnz], 0 <= col < n, no repeated column within a row
 *   val         double[nnz], finite
 *   row_sense   int8[m], AAPDHG_ROW_GE or AAPDHG_ROW_EQ
 *   q           double[m] (h and b of eq. lambda-case), finite
 *   c           double[n], finite
 *   lb, ub      double[n], lb <= ub, -INFINITY / +INFINITY allowed (eq. LP-O)
 *   precision   AAPDHG_FP64: iterates, SpMVs and reductions in FP64.
 *               AAPDHG_MIXED: K, iterates, SpMVs and the Anderson memory in
 *               FP32 with FP32 SpMV accumulation; Gram entries, the m x m
 *               solve, the safeguard test and the KKT norms accumulate to
 *               FP64 accuracy.
 *   mem_kind    AAPDHG_MEM_HOST: the arrays above are host memory.
 *               AAPDHG_MEM_DEVICE: they are device memory of the current device
 *               (read once, before this call returns).
 *   cuda_stream cudaStream_t for all work of the handle; NULL = a new
 *               non-blocking stream owned by the handle.
 *   out         receives the handle (NULL on error).
 * The problem is validated (AAPDHG_ERR_INVALID on a malformed CSR, a
 * non-finite value, lb > ub or an unknown sense) and copied to the device.
 * Defaults after create: AA-PDHG with m_A = 5, D = 10, eps = 1, eta = 1e-10,
 * beta = 1, c_s = 0.2, kappa = 1e8, c_div = 1, D-hat of the Remark, adaptive
 * FAA memory; no step sizes (aapdhg_iterate fails until they are set);
 * start x0 = P_X(0), y0 = 0.                                                  */
aapdhg_status aapdhg_create(int32_t m, int32_t n, int64_t nnz, const int64_t *row_ptr,
                            const int32_t *col_idx, const double *val, const int8_t *row_sense,
                            const double *q, const double *c, const double *lb, const double *ub,
                            int32_t precision, int32_t mem_kind, void *cuda_stream,
                            aapdhg_t *out);

/* Step sizes tau, sigma of eq. pdhg.  Both must be finite and > 0; the
 * convergence theory assumes sigma tau ||K||^2 < 1 (Assumption of Sec. 3),
 * which the caller establishes (e.g. with aapdhg_estimate_norm).  Resets the
 * run (as aapdhg_reset).                                                      */
aapdhg_status aapdhg_set_steps(aapdhg_t h, double tau, double sigma);

/* Estimate ||K||_2 by power iteration on K'K (the step-size rule of Sec. 5.1)
 * with `iters` iterations from a seeded start vector; writes the estimate to
 * *norm.  Uses the handle's stream and synchronises it.                       */
aapdhg_status aapdhg_estimate_norm(aapdhg_t h, int32_t iters, uint64_t seed, double *norm);

/* Method and Anderson parameters (Alg. 2 and Alg. 3-6):
 *   method      AAPDHG_PDHG, AAPDHG_AA (Alg. 2) or AAPDHG_FAA (Alg. 3)
 *   m_A         memory, 0 <= m_A <= AAPDHG_MAX_MEMORY (0: never accelerates)
 *   D, eps      safeguard ||g^k|| <= D ||g^0|| (i^k / c_div + 1)^-(1+eps), D > 0, eps > 0
 *   eta         Tikhonov parameter of Alg. 2 (>= 0; unused by FAA)
 *   beta        damping in (0, 1]
 *   c_s, kappa  angle / length filter thresholds of Alg. 4 / 5 (0 < c_s <= 1, kappa > 0)
 *   c_div       safeguard divisor >= 1 (1 is Alg. 2; 3 is the "Iter_AA / c" variant)
 *   dhat_mode   0: D-hat = I; 1: D-hat of the Remark on its construction
 *   faa_adaptive 1: columns removed by the filters leave the memory (the
 *               implemented variant of Sec. 5); 0: the filters act on a copy
 * Resets the run (as aapdhg_reset).                                           */
aapdhg_status aapdhg_set_method(aapdhg_t h, int32_t method, int32_t m_A, double D, double eps,
                                double eta, double beta, double c_s, double kappa, double c_div,
                                int32_t dhat_mode, int32_t faa_adaptive);

/* Diagonal preconditioning of the LP, the set-up of the paper's comparison
 * with restarted PDHG (Sec. 5.2: Ruiz scaling for 10 iterations combined with
 * the Pock-Chambolle technique).  Each of the ruiz_iters passes divides every
 * row and every column of the current scaled K by the square root of its
 * largest |entry|; pock_chambolle != 0 adds one pass that divides them by the
 * square root of their sum of |entries| (alpha = 1).  Empty rows and columns
 * keep factor 1.  With the products Dr (rows) and Dc (columns) the solver then
 * iterates on Dr K Dc, Dr q, Dc c and the bounds divided by Dc; start points
 * (aapdhg_set_start), iterates (aapdhg_get_iterate: x = Dc x~, y = Dr y~) and
 * the KKT quantities stay in the caller's units.  D-hat is formed from the
 * scaled K.  Runs on the device; may be applied once per handle
 * (AAPDHG_ERR_INVALID otherwise, or for ruiz_iters outside 0..1000); resets
 * the run.  Step sizes are the caller's: estimate them after scaling.        */
aapdhg_status aapdhg_set_scaling(aapdhg_t h, int32_t ruiz_iters, int32_t pock_chambolle);

/* Start point u^0 = (x0, y0) (host arrays of n and m doubles, or NULL for the
 * default x0 = P_X(0), y0 = 0).  The start is projected onto X x Y, as Alg. 2
 * asks for a feasible start.  Resets the run.                                 */
aapdhg_status aapdhg_set_start(aapdhg_t h, const double *x0, const double *y0);

/* Forget the run: the next aapdhg_iterate starts again from u^0 with an empty
 * Anderson memory and zero counters.                                          */
aapdhg_status aapdhg_reset(aapdhg_t h);

/* Run at most max_iters loop iterations of Alg. 2 / Alg. 3 (resumable: a
 * later call continues from the current iterate and memory).  The first call
 * after a reset also forms u^1 = T u^0 and g^0 (not counted as an iteration).
 * Every kkt_every-th iteration (counted over the whole run, first at
 * iteration 0; kkt_every <= 0 disables the test) the KKT residual of the
 * current iterate u^k is evaluated before T(u^k) is used; the run stops at u^k
 * when it is <= tol.  *iters_done (may be NULL) receives the iterations done
 * by this call.  Returns AAPDHG_OK when the tolerance was met (now or in an
 * earlier call), AAPDHG_NOT_CONVERGED when max_iters ran out, or an error.    */
aapdhg_status aapdhg_iterate(aapdhg_t h, int64_t max_iters, double tol, int32_t kkt_every,
                             int64_t *iters_done);

/* Time limit of the run, in seconds of wall-clock time spent in
 * aapdhg_iterate since the last reset (the numerical experiments of Sec. 5
 * stop every run at KKT <= 1e-4 or one hour); 0 (the default) switches it off.
 * aapdhg_iterate checks it between chunks of 64 iterations and, once it has
 * run out, returns AAPDHG_ERR_TIMEOUT with *iters_done set.  The status is not
 * sticky: the run stays at its last iterate and continues under a new limit.
 * seconds must be finite and >= 0 (AAPDHG_ERR_INVALID otherwise).           */
aapdhg_status aapdhg_set_time_limit(aapdhg_t h, double seconds);

/* Current iterate u^k: x (n doubles) and y (m doubles) in the caller's row and
 * column order; either pointer may be NULL.                                   */
aapdhg_status aapdhg_get_iterate(aapdhg_t h, double *x, double *y);

/* KKT quantities of the current iterate (Remark on termination conditions),
 * evaluated now: out[0..5] = {r_p, r_d, r_g, KKT, c'x, dual objective}, with
 * lambda = P_Lambda(c - K'y).                                                 */
aapdhg_status aapdhg_get_kkt(aapdhg_t h, double *out6);

/* Counters of the run: i (AA steps taken), j (PDHG steps taken), iterations,
 * and AA steps rejected because the m x m factorisation failed (counted in
 * j).  Any pointer may be NULL.                                               */
aapdhg_status aapdhg_get_counters(aapdhg_t h, int64_t *aa_steps, int64_t *pdhg_steps,
                                  int64_t *iters, int64_t *ls_failures);

/* Per-iteration trace for the first `capacity` iterations of the next run
 * (capacity 0 disables; resets the run).  aapdhg_get_trace copies up to
 * *len entries: branch (0 PDHG step, 1 AA step, 2 AA step rejected by a failed
 * factorisation), ||g^k||, KKT(u^k) (NaN when not evaluated) and the number
 * of memory columns used by an accepted AA step (-1 otherwise).  Any output
 * pointer may be NULL; *len receives the entries written.                     */
aapdhg_status aapdhg_set_trace(aapdhg_t h, int64_t capacity);
aapdhg_status aapdhg_get_trace(aapdhg_t h, int64_t *len, int8_t *branch, double *gnorm,
                               double *kkt, int32_t *mk);

/* Test hook: the Anderson memory of Alg. 2 as the device holds it after the
 * last iteration k (the columns of dG^{k-m_k} and their Gram matrix).
 * *count (optional) receives the number of columns c; gram (c x c, row-major) = <dg_a, dg_b> and rhs (c) = <dg_a, g^k>, columns oldest
 * first, as accumulated on the device (FP64, or float-float pairs summed in
 * FP64 in mixed mode).  The device forms a new column's entries with the
 * other columns, and the right-hand side, at the next AA attempt (an
 * iteration whose safeguard test passed): after an iteration without one,
 * the entries of the columns added since the last attempt, and rhs except
 * for the newest column, are pending (left as they were).  dg (c x (n + m),
 * column a at a * (n + m)) and g
 * (n + m) = g^k hold the stored vectors in the caller's variable then
 * constraint order, in the solver's units (scaled when aapdhg_set_scaling was
 * applied), FP32 values widened exactly in mixed mode.  Any output may be
 * NULL; capacity below c gives AAPDHG_ERR_INVALID (with *count set).  No
 * columns before the first iteration or for plain PDHG.                     */
aapdhg_status aapdhg_get_memory(aapdhg_t h, int32_t capacity, int32_t *count, double *gram,
                                double *rhs, double *dg, double *g);

/* Checkpoint / resume of a run (the paper has none; its experiments stop at a
 * time limit).  aapdhg_state_size gives the bytes of the handle's state blob;
 * aapdhg_get_state copies the blob into the caller's host buffer `buf` of
 * exactly that size: the run state on the device (the iterates u^k and
 * T(u^k) as pairs, g^k, D-hat, the two Anderson rings with the Gram matrix,
 * column list, counters i^k, j^k and the safeguard's g^0, the primal-weight
 * snapshot) and on the host (the step sizes and primal weight, the layouts,
 * the time used).  aapdhg_set_state restores a blob into a handle created
 * from the same LP in the same precision with the same set-up calls
 * (scaling, method and memory, primal weight period); it rebuilds the layouts
 * when they differ, so that every sum runs in the blob's order.  Iterating
 * after a restore gives bit for bit what the run the blob was taken from
 * gives.  The caller owns the buffer; nothing is kept.  A NULL buffer, a size
 * other than aapdhg_state_size (get) or the blob's own (set), a blob of
 * another LP, precision or set-up, or a corrupt header gives
 * AAPDHG_ERR_INVALID.                                                         */
aapdhg_status aapdhg_state_size(aapdhg_t h, size_t *bytes);
aapdhg_status aapdhg_get_state(aapdhg_t h, void *buf, size_t bytes);
aapdhg_status aapdhg_set_state(aapdhg_t h, const void *buf, size_t bytes);

/* Kernel instrumentation for benchmarks.  aapdhg_profile_kernels(h, 1) makes
 * aapdhg_iterate bracket every kernel it launches with CUDA events recorded on
 * the handle's stream and accumulate the elapsed times per kernel kind; it
 * resets the totals (0 turns the events off).  aapdhg_get_kernel_profile
 * returns, for kind 0 (x-step over K'), 1 (y-step over K), 2 (memory pass:
 * the new column, and the m x m work of an iteration without an AA attempt),
 * 3 (AA mix) or 4 (Gram pass and m x m solve of an AA attempt), the launches
 * and total milliseconds since the
 * last reset; kind -1 returns the number of kernels aapdhg_iterate launched
 * since create (counted with or without events) and 0 ms.                    */
aapdhg_status aapdhg_profile_kernels(aapdhg_t h, int32_t enable);
aapdhg_status aapdhg_get_kernel_profile(aapdhg_t h, int32_t kind, int64_t *launches,
                                        double *total_ms);

/* Primal weight update with memory reset and D-hat re-blend (Alg. "Primal
 * weight update" and the Remark on its form).  period = U_P > 0 switches it
 * on: the given steps define gamma = sqrt(tau sigma) and omega^0 =
 * sqrt(sigma / tau); when the current iterate is u^k with k > 0, k = 0 mod
 * U_P, Delta_x = ||x^k - x^{k-U_P}|| and Delta_y likewise, and if both exceed
 * eps_zero: omega <- exp(theta log(Delta_y/Delta_x) + (1 - theta) log omega),
 * tau = gamma / omega, sigma = gamma omega, the Anderson memory is reset (that
 * iteration takes the plain step), and with dhat_blend = 1 D-hat <-
 * (1 - alpha) diag(1/omega, omega) + alpha diag(D1/omega, D2 omega), alpha =
 * alpha_dec when the relative decrease of ||g|| over the last iteration is
 * >= rho_min, else alpha_inc (paper: alpha 0.1 / 0.9, theta 0.5, U_P 3000).
 * period = 0 switches it off.  With FP32 iterates (AAPDHG_MIXED) and
 * kkt_every > 0 an update is applied only while the run still improves: the
 * last KKT test must be below every KKT seen at the earlier update points
 * (at FP32's attainable accuracy the Deltas are rounding noise and omega
 * would drift; FP64 applies every update, as the paper).  theta, alpha_* in
 * [0, 1], eps_zero >= 0 (AAPDHG_ERR_INVALID otherwise).  Resets the run.    */
aapdhg_status aapdhg_set_primal_weight(aapdhg_t h, int64_t period, double theta, double eps_zero,
                                       int32_t dhat_blend, double rho_min, double alpha_dec,
                                       double alpha_inc);

/* Autotuning of the two PDHG half-step kernels (the SpMVs of eq. pdhg; the
 * paper has no counterpart).  They are compiled for AAPDHG_TASK_SHAPES task
 * shapes (shape 0: two SELL slices per warp task, 8 loads in flight per lane;
 * 1: one slice, 8 loads; 2: four slices, 8 loads; 3: one slice, 16 loads;
 * 4: two slices, 16 loads), which sum every row in the
 * same order, so the shape never changes a result.  By default the first
 * aapdhg_iterate times every shape on the handle's matrices and keeps the
 * fastest of each kernel.  aapdhg_autotune does that now and returns the
 * chosen shapes and (avg_us, optional: 2 * AAPDHG_TASK_SHAPES doubles, x-step
 * shapes then y-step shapes) the average launch time of each; it changes no
 * run state.  aapdhg_set_task_shape fixes the two shapes (no tuning), or with
 * (-1, -1) re-enables tuning at the next iterate; other values give
 * AAPDHG_ERR_INVALID.                                                        */
enum { AAPDHG_TASK_SHAPES = 5 };
aapdhg_status aapdhg_autotune(aapdhg_t h, int32_t *shape_x, int32_t *shape_y, double *avg_us);
aapdhg_status aapdhg_set_task_shape(aapdhg_t h, int32_t shape_x, int32_t shape_y);

/* Layouts of the two half-steps' matrices K' and K (the SpMVs of eq. pdhg;
 * the paper has no counterpart).  Rows are numbered longest first; rows of at
 * most sell_max entries are stored in SELL-32 slices and read one lane per
 * row; longer rows are cut into chunks of long_chunk entries, one warp per
 * chunk (32 lanes per row).  The default is sell_max = 32, long_chunk = 1024
 * for both matrices.  aapdhg_set_layout rebuilds both layouts from layout4 =
 * {sell_max, long_chunk of K' (the x-step), sell_max, long_chunk of K (the
 * y-step)}, from the matrices on the device (as scaled), and keeps the run
 * state; the task shapes are tuned again at the next iterate.  1 <= sell_max
 * <= 1024, long_chunk a multiple of 32 in [32, 2^20] (AAPDHG_ERR_INVALID
 * otherwise).  A row's sum runs in a different order under another layout,
 * so results change by rounding only.  aapdhg_autotune_layout builds each of
 * AAPDHG_LAYOUT_CANDIDATES layouts in turn for both matrices ((sell_max,
 * long_chunk) = (32, 1024), (16, 1024), (64, 1024), (128, 1024), (32, 2048),
 * (64, 2048), (128, 2048), (64, 4096)), tunes the task shapes on it, and keeps
 * for K' the candidate with the fastest x-step and for K the one with the
 * fastest y-step; it returns the choice in layout4 (optional) and, in avg_us
 * (optional, 2 * AAPDHG_LAYOUT_CANDIDATES doubles), the best x-step and
 * y-step launch time of each candidate.  It changes no run state; it is not
 * run by aapdhg_iterate.                                                     */
enum { AAPDHG_LAYOUT_CANDIDATES = 8 };
aapdhg_status aapdhg_set_layout(aapdhg_t h, const int32_t *layout4);
aapdhg_status aapdhg_autotune_layout(aapdhg_t h, int32_t *layout4, double *avg_us);

/* KKT residuals of a given point without any device allocation.  The paper
 * has no counterpart to this entry point.  It exists for callers that cannot
 * allocate device memory when they need the residuals: latency-critical loops
 * that must not hit the implicit device synchronisation of cudaMalloc /
 * cudaFree, and programs whose device memory is owned by another framework's
 * pool or a fixed budget, where an allocation of the library's own would fail
 * or fragment that pool.  Its scratch (block partial sums and an arrival
 * counter) is a fixed file-scope device array of
 * AAPDHG_NOALLOC_MAX_BLOCKS * 8 doubles (1 MiB), held by every GPU that loads
 * the library until the process exits.
 *
 * Inputs, all device memory of the current device, caller-owned, FP64 where
 * real-valued, in the caller's row and column order:
 *   m, n                      rows of K and variables (n >= 1)
 *   row_ptr/col_idx/val       K = [G; A] as CSR (int64 row pointers, int32 columns)
 *   t_row_ptr/t_col_idx/t_val K' as CSR (n rows)
 *   row_sense, q, c, lb, ub   as in aapdhg_create
 *   x (n), y (m)              the point
 * Output: out6 (device, 6 doubles) = {r_p, r_d, r_g, KKT, c'x, dual objective},
 * the quantities of aapdhg_get_kkt, written on cuda_stream (NULL = legacy
 * default stream).  The call is asynchronous; it only checks arguments and
 * enqueues work.
 * Limits and errors: returns AAPDHG_ERR_INVALID without touching the device
 * when ceil(n / 512) + ceil(m / 512) > AAPDHG_NOALLOC_MAX_BLOCKS (about 8.4M
 * rows in total), when m < 0 or n < 1, or when a required pointer is NULL
 * (row_ptr, t_row_ptr, c, lb, ub, x and out6 always; col_idx, val, t_col_idx,
 * t_val, row_sense, q and y when m > 0); AAPDHG_ERR_CUDA when the scratch
 * address cannot be resolved or the launch fails.  aapdhg_last_error does not
 * report this entry point.
 * Set-up: the first call on each device resolves the scratch array's device
 * address (cudaGetSymbolAddress) with that device current and keeps it for
 * later calls; make that first call before any stream capture.  The kept
 * address belongs to the device's primary context, so calling this entry
 * point after a cudaDeviceReset of that device is not supported.  Calls
 * share the one scratch array: two calls whose work overlaps on the same GPU
 * (different streams, or graphs launched concurrently) race and give wrong
 * results; each call clears the counter it needs before its kernel starts.  */
enum { AAPDHG_NOALLOC_MAX_BLOCKS = 16384 };
aapdhg_status aapdhg_kkt_noalloc(int32_t m, int32_t n, const int64_t *row_ptr,
                                 const int32_t *col_idx, const double *val,
                                 const int64_t *t_row_ptr, const int32_t *t_col_idx,
                                 const double *t_val, const int8_t *row_sense, const double *q,
                                 const double *c, const double *lb, const double *ub,
                                 const double *x, const double *y, double *out6,
                                 void *cuda_stream);

/* Bytes of device memory held by the handle.                                 */
aapdhg_status aapdhg_device_bytes(aapdhg_t h, int64_t *bytes);

/* Message of the last error of the handle (or of the last failed create when
 * h is NULL).  The string lives until the next call on the handle.            */
const char *aapdhg_last_error(aapdhg_t h);

/* Free the handle and its device memory (synchronises its stream).          */
void aapdhg_destroy(aapdhg_t h);

/* ===========================================================================
 * Batched solver: many independent LPs advanced together on one GPU.
 *
 * The same method as above (PDHG step of eq. pdhg, Alg. 2 / Alg. 3 with the
 * safeguard, the termination test of the Remark on termination conditions),
 * applied to every LP of the batch at once; each LP has its own step sizes,
 * Anderson memory, safeguard, iteration count and stop flag, and stops when
 * its own KKT residual meets the tolerance.  The paper solves one LP at a
 * time; the batch packs the LPs into one block-diagonal LP (padded so each
 * problem's variable and constraint ranges start on 16-byte boundaries) and
 * computes every row of T(u) exactly as the single-LP solver does for that LP.
 * Method settings (aapdhg_batch_set_method) apply to all problems.
 *
 * Inputs of create are host memory, every per-problem array concatenated in
 * problem order:
 *   nprob                 number of LPs, 1 <= nprob < 2^25
 *   m[p], n[p], nnz[p]    sizes of LP p (as in aapdhg_create)
 *   row_ptr               sum(m[p] + 1) int64: each LP's own CSR row pointers
 *                         (starting at 0)
 *   col_idx, val          sum(nnz[p]): each LP's column indices (its own
 *                         variable numbering) and values
 *   row_sense, q          sum(m[p]);   c, lb, ub   sum(n[p])
 * Each LP is validated as aapdhg_create does (the error message names the
 * problem).  The packed batch must hold < 2^31 nonzeros and < 2^31 elements.
 * The library copies everything; the caller keeps ownership.  Defaults, the
 * allocator and the stream rules are those of aapdhg_create; the handle is
 * used from one host thread at a time.  Errors are sticky as for aapdhg_t,
 * except AAPDHG_ERR_NUMERIC from iterate, which reports that at least one LP
 * stopped on NaN/Inf while the others went on (see aapdhg_batch_get_status). */
typedef struct aapdhg_batch_s *aapdhg_batch_t;

aapdhg_status aapdhg_batch_create(int32_t nprob, const int32_t *m, const int32_t *n,
                                  const int64_t *nnz, const int64_t *row_ptr,
                                  const int32_t *col_idx, const double *val,
                                  const int8_t *row_sense, const double *q, const double *c,
                                  const double *lb, const double *ub, int32_t precision,
                                  void *cuda_stream, aapdhg_batch_t *out);

/* Per-problem step sizes tau[p], sigma[p] (host arrays of nprob, finite, > 0);
 * resets every problem to its start.                                         */
aapdhg_status aapdhg_batch_set_steps(aapdhg_batch_t h, const double *tau, const double *sigma);

/* Per-problem estimate of ||K_p||_2 by `iters` power iterations on K_p'K_p
 * (Sec. 5.1), all problems at once; norms: host array of nprob.  For a given
 * seed each problem starts from the vector the single-LP solver uses.        */
aapdhg_status aapdhg_batch_estimate_norms(aapdhg_batch_t h, int32_t iters, uint64_t seed,
                                          double *norms);

/* As aapdhg_set_method, for every problem of the batch.                      */
aapdhg_status aapdhg_batch_set_method(aapdhg_batch_t h, int32_t method, int32_t m_A, double D,
                                      double eps, double eta, double beta, double c_s,
                                      double kappa, double c_div, int32_t dhat_mode,
                                      int32_t faa_adaptive);

/* As aapdhg_set_scaling, each problem scaled on its own rows and columns.    */
aapdhg_status aapdhg_batch_set_scaling(aapdhg_batch_t h, int32_t ruiz_iters, int32_t pock_chambolle);

/* As aapdhg_set_primal_weight, for every problem of the batch on its own:
 * each problem's gamma and omega^0 come from its own steps, and at every
 * batch iterate u^k with k = 0 mod U_P each running problem measures its own
 * Delta_x, Delta_y, and updates its own omega, steps, D-hat and memory (or
 * leaves them when a Delta is <= eps_zero).  The update runs on the device
 * (no host round trip; aapdhg_batch_launch stays asynchronous).  A problem
 * that stops at the update iterate keeps that iterate.  Same parameter
 * ranges and errors as aapdhg_set_primal_weight.  Resets the run.          */
aapdhg_status aapdhg_batch_set_primal_weight(aapdhg_batch_t h, int64_t period, double theta,
                                             double eps_zero, int32_t dhat_blend, double rho_min,
                                             double alpha_dec, double alpha_inc);

/* Starts of all problems (concatenated caller-order x0: sum(n[p]), y0:
 * sum(m[p]); NULL = zeros), projected as in aapdhg_set_start; resets.        */
aapdhg_status aapdhg_batch_set_start(aapdhg_batch_t h, const double *x0, const double *y0);
aapdhg_status aapdhg_batch_reset(aapdhg_batch_t h);

/* Run up to max_iters batch iterations (the first call also forms u^1 = T u^0
 * of every problem first, as aapdhg_iterate does).  A problem's KKT residual
 * is tested every kkt_every iterations (0: never); a problem stops when it is
 * <= tol and is left unchanged from then on; the call returns early when every
 * problem has stopped.  iters_done (optional): batch iterations run by this
 * call.  A new call re-tests every converged problem against its tolerance.
 * Returns AAPDHG_OK when every problem met the tolerance, AAPDHG_NOT_CONVERGED
 * when max_iters ran out first, AAPDHG_ERR_NUMERIC (not sticky) when some
 * problem stopped on NaN/Inf, or an error.                                   */
aapdhg_status aapdhg_batch_iterate(aapdhg_batch_t h, int64_t max_iters, double tol,
                                   int32_t kkt_every, int64_t *iters_done);

/* Per-problem tolerances (host array of nprob, each >= 0): problem p stops
 * when its KKT residual is <= tol[p]; the tol argument of iterate / launch is
 * then ignored.  NULL restores one tolerance for all.                        */
aapdhg_status aapdhg_batch_set_tolerances(aapdhg_batch_t h, const double *tol);

/* Asynchronous form of iterate: aapdhg_batch_launch enqueues n_iters batch
 * iterations on the handle's stream and returns without waiting (the first
 * call after create / reset / a set_* call also forms u^1 = T u^0 of every
 * problem first).  Unlike iterate it does not re-test problems that already
 * converged.  aapdhg_batch_poll waits for the enqueued work, reads every
 * problem's state (then available through aapdhg_batch_get_status) and sets
 * *all_stopped (optional) to 1 when every problem has converged or failed.    */
aapdhg_status aapdhg_batch_launch(aapdhg_batch_t h, int64_t n_iters, double tol, int32_t kkt_every);
aapdhg_status aapdhg_batch_poll(aapdhg_batch_t h, int32_t *all_stopped);

/* Current iterates of all problems in the caller's order, concatenated as the
 * inputs (x: sum(n[p]), y: sum(m[p]); either may be NULL).                   */
aapdhg_status aapdhg_batch_get_iterate(aapdhg_batch_t h, double *x, double *y);

/* One problem's current iterate (x: n[p], y: m[p], its caller order), the KKT
 * quantities of its last test (kkt6, as aapdhg_get_kkt; all 0 before the
 * first test) and its status row (status6, as aapdhg_batch_get_status), read
 * from that problem's ranges only; any output may be NULL.  A problem that
 * stopped keeps its iterate, so this can hand its result back while the others
 * run (after aapdhg_batch_poll).  p outside 0 .. nprob - 1: AAPDHG_ERR_INVALID. */
aapdhg_status aapdhg_batch_get_member(aapdhg_batch_t h, int32_t p, double *x, double *y,
                                      double *kkt6, int64_t *status6);

/* KKT quantities of every problem's current iterate: out6[6p .. 6p+5] as in
 * aapdhg_get_kkt (host array of 6 * nprob).                                  */
aapdhg_status aapdhg_batch_get_kkt(aapdhg_batch_t h, double *out6);

/* Per-problem status, out6[6p .. 6p+5] = {iterations, AA steps, PDHG steps,
 * factorisation failures, converged (0/1), NaN/Inf met (0/1)}.               */
aapdhg_status aapdhg_batch_get_status(aapdhg_batch_t h, int64_t *out6);

/* CUDA-event timing of the batch kernels by kind: 0 half-step x, 1 half-step
 * y, 2 memory pass, 3 AA mix, 4 per-problem KKT, 5 per-problem push and
 * safeguard, Gram pass and m x m work of the attempts; kind -1 gives in *launches
 * the number of kernels launched since profiling was last (re)set.          */
aapdhg_status aapdhg_batch_profile_kernels(aapdhg_batch_t h, int32_t enable);
aapdhg_status aapdhg_batch_get_kernel_profile(aapdhg_batch_t h, int32_t kind, int64_t *launches,
                                              double *total_ms);

/* As aapdhg_autotune / aapdhg_set_task_shape, on the packed batch.          */
aapdhg_status aapdhg_batch_autotune(aapdhg_batch_t h, int32_t *shape_x, int32_t *shape_y,
                                    double *avg_us);
aapdhg_status aapdhg_batch_set_task_shape(aapdhg_batch_t h, int32_t shape_x, int32_t shape_y);

/* As aapdhg_set_layout / aapdhg_autotune_layout, on the packed batch: the
 * layouts of the packed K' and K are rebuilt from the matrices on the device,
 * every problem's rows in their own slices and chunks (so a problem's sums
 * depend on the layout parameters only, not on the other problems), with the
 * run state kept.  The default is (32, 1024) for both matrices.             */
aapdhg_status aapdhg_batch_set_layout(aapdhg_batch_t h, const int32_t *layout4);
aapdhg_status aapdhg_batch_autotune_layout(aapdhg_batch_t h, int32_t *layout4, double *avg_us);

aapdhg_status aapdhg_batch_device_bytes(aapdhg_batch_t h, int64_t *bytes);
const char *aapdhg_batch_last_error(aapdhg_batch_t h);
void aapdhg_batch_destroy(aapdhg_batch_t h);

/* ===========================================================================
 * Served stream: LPs arriving over time, solved with continuous batching.
 *
 * A server admits submitted LPs, as the device memory budget allows, into
 * cohorts (batched solvers, each on its own CUDA stream) and advances all
 * cohorts together, one chunk of kkt_every = 64 iterations per cohort per
 * aapdhg_server_step.  Every cohort is set up as Sec. 5 describes (Ruiz x10 +
 * Pock-Chambolle scaling, step sizes 0.9 / ||K_p|| from 100 power iterations,
 * the given method and memory, D = 10, eps = 1, eta = 1e-10, beta = 1,
 * c_s = 0.2, kappa = 1e8), each LP with its own tolerance; LPs whose tolerance
 * is below 1e-5 are solved in FP64 cohorts, the others in mixed precision.
 * An LP that converged or failed has its result handed back by the step that
 * observes it (its state and result are then final), while the rest of its
 * cohort runs on; the cohort's memory is freed when every member has finished
 * (converged, failed or at the iteration cap).  The paper solves one LP at a
 * time; this is its method applied to a stream.
 *
 *   create:  method, m_A as aapdhg_set_method; max_cohorts >= 1 running at
 *            once; max_cohort_size >= 1 LPs per cohort; max_iters >= 1 per
 *            LP; mem_budget device bytes all cohorts may hold (0: 80% of the
 *            free device memory at create).
 *   submit:  one LP in the form of aapdhg_create (host memory, copied), tol > 0;
 *            returns its id.  A malformed LP (the checks of aapdhg_create) is
 *            refused with AAPDHG_ERR_INVALID, which is not sticky; an LP larger
 *            than the whole budget ends in state AAPDHG_REQ_REJECTED.
 *   step:    one scheduling round (launch, admit, poll, retire); *running and
 *            *waiting (optional) give the cohorts on the GPU and the LPs
 *            queued after the round.
 *   result:  state of LP `id`; times3 (optional) = {submit, admit, done} in
 *            seconds from create (-1: not yet); x (n), y (m), kkt6 (as
 *            aapdhg_get_kkt) and iters once the state is CONVERGED, CAPPED or
 *            ERROR after admission.
 * The server and its cohorts are used from one host thread.                  */
typedef struct aapdhg_server_s *aapdhg_server_t;
enum {
    AAPDHG_REQ_WAITING = 0, AAPDHG_REQ_RUNNING = 1, AAPDHG_REQ_CONVERGED = 2,
    AAPDHG_REQ_CAPPED = 3, AAPDHG_REQ_ERROR = 4, AAPDHG_REQ_REJECTED = 5
};
aapdhg_status aapdhg_server_create(int32_t method, int32_t m_A, int32_t max_cohorts,
                                   int32_t max_cohort_size, int64_t max_iters,
                                   int64_t mem_budget, aapdhg_server_t *out);
aapdhg_status aapdhg_server_submit(aapdhg_server_t s, int32_t m, int32_t n, int64_t nnz,
                                   const int64_t *row_ptr, const int32_t *col_idx,
                                   const double *val, const int8_t *row_sense, const double *q,
                                   const double *c, const double *lb, const double *ub, double tol,
                                   int64_t *id);
/* Primal weight update (as aapdhg_batch_set_primal_weight) for the cohorts
 * admitted after the call; period 0 switches it off for them.  Parameters out
 * of range: AAPDHG_ERR_INVALID, not sticky.                                 */
aapdhg_status aapdhg_server_set_primal_weight(aapdhg_server_t s, int64_t period, double theta,
                                              double eps_zero, int32_t dhat_blend, double rho_min,
                                              double alpha_dec, double alpha_inc);
aapdhg_status aapdhg_server_step(aapdhg_server_t s, int32_t *running, int32_t *waiting);
aapdhg_status aapdhg_server_result(aapdhg_server_t s, int64_t id, int32_t *state, double *x,
                                   double *y, double *kkt6, int64_t *iters, double *times3);
aapdhg_status aapdhg_server_device_bytes(aapdhg_server_t s, int64_t *bytes);
const char *aapdhg_server_last_error(aapdhg_server_t s);
void aapdhg_server_destroy(aapdhg_server_t s);

#ifdef __cplusplus
}
#endif
#endif /* AAPDHG_H */
