/*
 * rhpdhg.h -- C ABI of a single-GPU (sm_103a) solver for linear programs by restarted Halpern
 * PDHG (rHPDHG) and reflected restarted Halpern PDHG (r2HPDHG), after H. Lu and J. Yang,
 * "Restarted Halpern PDHG for Linear Programming" (arXiv 2407.16144).
 *
 * Problem (general form; the paper's eq. lp, Section 2, is the case m_ineq = 0, l = 0, u = +inf):
 *
 *     minimize    c^T x + obj_offset
 *     subject to  A x  = b        rows 0 .. m_eq-1 of K
 *                 G x >= h        rows m_eq .. m_eq+m_ineq-1 of K
 *                 l <= x <= u     entries of l may be -INFINITY, entries of u +INFINITY
 *
 * K = [A; G] is given in CSR; rhs = [b; h].  The method iterates the PDHG operator T of
 * eq. pdhg (Section 2) inside the Halpern scheme of eq. hpdhg (Algorithm 1) or of its reflected
 * form eq. hrpdhg (Algorithm 2), restarting by the fixed-point-residual rule of
 * eq. adaptive-restart (Section 3).  The dual variable y follows the Lagrangian sign
 * L(x, y) = c^T x - y^T (K x - rhs): y equals the paper's y of eq. pdhg with its sign flipped, so
 * y >= 0 on the G rows.
 *
 * Conventions shared by every function below:
 *   - Return value: RHPDHG_OK (0) on success, RHPDHG_BUSY (1) from poll while a solve is still
 *     running, a negative RHPDHG_ERR_* code on failure.  rhpdhg_last_error() gives the message.
 *     No function aborts, exits or traps; a device-side wait that runs out of its bound reports
 *     RHPDHG_ERR_DEVICE_TIMEOUT.
 *   - Problem outcomes (optimal, infeasible, limits) are statuses in rhpdhg_result, not errors.
 *   - Ownership: create() copies every input, so the caller may free its arrays afterwards.
 *     Output arrays in rhpdhg_result are owned by the caller and written by poll().
 *   - A handle is used by one host thread at a time.
 */
#ifndef RHPDHG_H
#define RHPDHG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------------------------- */
#define RHPDHG_OK                  0
#define RHPDHG_BUSY                1
#define RHPDHG_ERR_INVALID_ARG    -1   /* malformed CSR, NaN data, l > u, bad parameter        */
#define RHPDHG_ERR_OOM            -2   /* device or pinned-host allocation failed              */
#define RHPDHG_ERR_CUDA           -3   /* a CUDA runtime call failed                           */
#define RHPDHG_ERR_DEVICE_TIMEOUT -4   /* a bounded device-side wait ran out                   */
#define RHPDHG_ERR_STATE          -5   /* call not valid in the handle's current state         */

/* ---- solve statuses (rhpdhg_result.status) ---------------------------------------------- */
#define RHPDHG_STATUS_RUNNING            0
#define RHPDHG_STATUS_OPTIMAL            1   /* rel-KKT <= eps_rel_kkt at the returned point   */
#define RHPDHG_STATUS_PRIMAL_INFEASIBLE  2   /* cert_y holds a Farkas vector                   */
#define RHPDHG_STATUS_DUAL_INFEASIBLE    3   /* cert_x holds an unbounded primal ray           */
#define RHPDHG_STATUS_ITERATION_LIMIT    4
#define RHPDHG_STATUS_TIME_LIMIT         5
#define RHPDHG_STATUS_NUMERICAL_ERROR    6   /* a residual norm became NaN or infinite         */
#define RHPDHG_STATUS_CANCELLED          7

/* ---- certificate sources (rhpdhg_result.cert_source) ------------------------------------ */
/* The two certificate candidates are the limits of Lemma sublinear-infeas that Theorem infeas
 * carries over to restarts: the displacement T(z) - z (tested at every restart point z^{n,0},
 * n >= 1, and at every check iteration) and the anchor movement z^{n+1,0} - z^{n,0} (tested at
 * every restart).  The first that passes the Farkas test is returned. */
#define RHPDHG_CERT_NONE            0
#define RHPDHG_CERT_RESTART_POINT   1   /* T(z) - z at a restart point                     */
#define RHPDHG_CERT_CHECK           2   /* T(z) - z at a check iteration                   */
#define RHPDHG_CERT_ANCHOR_MOVE     3   /* z^{n+1,0} - z^{n,0}                              */

/* ---- memory kinds ---------------------------------------------------------------------- */
#define RHPDHG_MEM_HOST    0
#define RHPDHG_MEM_DEVICE  1

typedef struct rhpdhg_handle rhpdhg_handle;

/* The LP.  All arrays are read during rhpdhg_create only.
 *   memory:  RHPDHG_MEM_HOST (pageable or pinned host memory) or RHPDHG_MEM_DEVICE (device
 *            memory of the current device).
 *   row_ptr: m+1 non-decreasing offsets, row_ptr[0] = 0, row_ptr[m] = nnz.
 *   col_idx: nnz column indices in [0, n), strictly increasing within each row.
 *   val:     nnz finite values.
 *   c, l, u: n entries; rhs: m entries (b then h).  l <= u; l may hold -INFINITY and u
 *            +INFINITY; c and rhs finite.
 * Validation of the CSR structure and of the data (NaN, l > u) is done on the host for host
 * memory and on the device for device memory; failures return RHPDHG_ERR_INVALID_ARG.        */
typedef struct {
  int32_t m_eq;
  int32_t m_ineq;
  int32_t n;
  int32_t memory;
  int64_t nnz;
  const int64_t *row_ptr;
  const int32_t *col_idx;
  const double  *val;
  const double  *c;
  const double  *rhs;
  const double  *l;
  const double  *u;
  double obj_offset;
} rhpdhg_problem;

/* A caller's device allocator (for instance a framework's caching allocator), used by
 * rhpdhg_create for every device buffer of the handle and for its own temporaries.  alloc
 * returns `bytes` of device memory of the current device, aligned to 256 bytes, usable on
 * cuda_stream (the handle's stream), or NULL when it cannot; free takes back a pointer alloc
 * returned, with the same stream and ctx.  The library calls free only when no work on the
 * buffer is pending, from the thread that calls rhpdhg_free (or rhpdhg_create, on failure). */
typedef void *(*rhpdhg_dev_alloc_fn)(size_t bytes, void *cuda_stream, void *ctx);
typedef void (*rhpdhg_dev_free_fn)(void *ptr, void *cuda_stream, void *ctx);

/* Algorithm parameters.  rhpdhg_params_default() fills the documented defaults. */
typedef struct {
  int32_t algorithm;            /* 0 = rHPDHG (Algorithm 1, eq. hpdhg); 1 = r2HPDHG
                                   (Algorithm 2, eq. hrpdhg).                        default 1 */
  int32_t precision;            /* 0 = FP64 throughout; 1 = FP32 matrix values and iterates with
                                   FP64 anchors, restarts, residuals and checks.  When a
                                   certificate candidate comes within 1e-3 of the Farkas test at
                                   two restart points in a row, the solve continues in FP64 from
                                   the second (iterations and epochs carry on); 2 = as 1 with
                                   BF16 matrix values: the scaling factors are rounded to powers
                                   of two, so K^ = D K E is exact in BF16 when every value of K
                                   has at most 8 significant bits (small integers such as the
                                   +-1 of an incidence matrix); otherwise create fails with
                                   RHPDHG_ERR_INVALID_ARG.  Precision 2 takes df_sums = 0.
                                                                                  default 0 */
  double  eps_rel_kkt;          /* stop when max(rel_p, rel_d, rel_gap) <= eps.   default 1e-4  */
  double  eps_infeas;           /* certificate tolerance (normalised violation).  default 1e-8  */
  int64_t max_iters;            /* PDHG evaluations T(z).                         default 1e7   */
  double  time_limit_s;         /* wall clock, checked between graph launches.    default 3600  */
  int32_t ruiz_iters;           /* Ruiz infinity-norm equilibration passes.       default 10    */
  double  pock_chambolle_alpha; /* Pock-Chambolle exponent; < 0 skips the pass.   default 1.0   */
  double  step_size;            /* eta; 0 = step_safety / sigma_max(K^) from power iteration */
  double  step_safety;          /*                                                default 0.9   */
  int32_t power_iters;          /* power-iteration steps for sigma_max.           default 100   */
  double  primal_weight;        /* omega_0; 0 = ||c^|| / ||rhs^|| (1 if either is ~0)           */
  int32_t primal_weight_update; /* 1 = omega <- exp(0.5 log(dy/dx) + 0.5 log omega) at restarts */
  int32_t first_epoch_len;      /* tau^0 of eq. adaptive-restart (restart once k > tau^0 in the
                                   first epoch).                                  default 64    */
  int64_t max_epoch_len;        /* restart once k >= this (0 = no cap).           default 1000  */
  int32_t restart_scheme;       /* 0 = adaptive (eq. adaptive-restart); 1 = fixed frequency
                                   every max_epoch_len (eq. fixed-restart); 2 = two-phase (the
                                   remark after Theorem infeas): the first epoch restarts once
                                   k >= first_epoch_len, every later one once k >= max_epoch_len.
                                   Schemes 1 and 2 need max_epoch_len >= 1.       default 0     */
  double  restart_beta;         /* restart when FPR <= beta * FPR(z^{n,0}).       default e^-1  */
  int32_t check_every;          /* termination-check cadence C (iterations).      default 64    */
  int32_t use_graphs;           /* 1 = replay a captured CUDA graph of C iterations. default 1  */
  int32_t trace;                /* 1 = record one rhpdhg_trace_rec per iteration (device).     */
  int32_t profile;              /* 1 = time the two per-iteration kernels with CUDA events
                                   (disables graphs); read with rhpdhg_kernel_times().        */
  int64_t trace_capacity;       /* records kept when trace = 1.                   default 4096  */
  const double *x0;             /* optional warm start, host memory, unscaled (n)  (Algorithm 1
                                   input z^{0,0}); NULL = projection of 0 onto [l, u]          */
  const double *y0;             /* optional warm start, host memory (m); NULL = 0              */
  int32_t adaptive_step;        /* 1 = the adaptive step rule (Section 7 adopts cuPDLP's): a step
                                   eta is accepted while eta <= ||dz||_w^2 / (2 |dy^T K dx|), the
                                   next one is min((1 - j^-0.3) eta_bar, (1 + j^-0.6) eta) with
                                   j = iteration + 2, and a rejected step is redone with it.
                                   precision 0 only; not in batched slots.       default 0    */
  int32_t cta_warps;            /* warps per CTA of the iteration kernels: 4, 8 or 16; 0 = the
                                   library's choice.                              default 0    */
  int32_t df_sums;              /* precision 1: sums of the restart test's norms (Section 3,
                                   eq. adaptive-restart) in ordinary iterations.  0 = FP32 sums of
                                   the FP32 products at every level (lane, warp, CTA, grid; fixed
                                   trees and orders); 1 = double-float (two FP32 numbers,
                                   error-free transformations) from the row up: FP64-grade sums,
                                   slower on GPUs with a narrow FP64 pipe.  Restart points always
                                   sum in FP64.                                   default 0    */
  /* Caller's allocator for the handle's device memory (both functions or neither; NULL = the
   * library's own cache of device buffers), with its context pointer.  Used by rhpdhg_create
   * only; the batched solver and the server ignore it.                          default NULL */
  rhpdhg_dev_alloc_fn dev_alloc;
  rhpdhg_dev_free_fn  dev_free;
  void *alloc_ctx;
  int32_t autotune;             /* 1 = rhpdhg_create times candidate launch shapes of the
                                   iteration kernels on the handle's stream and keeps the fastest
                                   per side: 4- or 8-warp CTAs; 1, 2 or 4 short tiles per work
                                   item where the group fits the staging area; plain or wide
                                   staging walk of the mixed row kernel; the full resident grid or
                                   three quarters of it.  The choice is cached for the process by
                                   a signature of the LP's structure (sizes, precision, algorithm,
                                   sum mode, row-length histograms), so handles of the same shape
                                   reuse it without timing.  Ignored when cta_warps or tile_mult
                                   is set.                                        default 0    */
  int32_t pow2_scaling;         /* 1 = the diagonal scalings D and E (Ruiz, then Pock-Chambolle)
                                   rounded to the nearest powers of two (a preconditioner that
                                   only shifts exponents; implied by precision 2). default 0   */
  int32_t tile_mult;            /* 0 = short tiles per work item by the layout rule (or the
                                   autotuner); 1, 2 or 4 = that many on each side whose longest
                                   group of tiles fits the staging area (other sides keep the
                                   rule).  rhpdhg_get_layout reports what each side walks.
                                                                                  default 0    */
} rhpdhg_params;

/* Result of a finished solve, filled by rhpdhg_poll. */
typedef struct {
  int32_t status;               /* RHPDHG_STATUS_*                                             */
  int32_t out_memory;           /* memory kind of x, y, cert_x, cert_y below (input to poll)   */
  int32_t cert_source;          /* RHPDHG_CERT_*: candidate behind an infeasibility status     */
  int32_t escalated;            /* precision 1 or 2: 1 if the solve continued in FP64 from a
                                   restart point (a near-certificate at two restart points in a
                                   row), else 0                                                 */
  int64_t iters;                /* PDHG evaluations performed                                  */
  int64_t restarts;             /* outer iterations n (restarts performed)                     */
  double  rel_p, rel_d, rel_gap;/* relative KKT parts at the returned point (last check)       */
  double  primal_obj, dual_obj;
  double  solve_seconds;        /* host wall clock from solve() to the final status           */
  double  eta, omega, sigma_max;/* step size (the last one with the adaptive rule), final
                                   primal weight, power-iteration estimate                    */
  double *x;                    /* caller-owned, n entries, or NULL: primal point (unscaled)   */
  double *y;                    /* caller-owned, m entries, or NULL: dual point (unscaled)     */
  double *cert_x;               /* caller-owned, n, or NULL: unbounded ray d (DUAL_INFEASIBLE) */
  double *cert_y;               /* caller-owned, m, or NULL: Farkas y (PRIMAL_INFEASIBLE)      */
} rhpdhg_result;

/* One per-iteration record (params.trace = 1). */
typedef struct {
  int64_t t;                    /* iteration (PDHG evaluation) index                           */
  int64_t epoch;                /* outer counter n                                             */
  int64_t k;                    /* inner counter k of the iterate z^{n,k}                      */
  double  fpr_sq;               /* ||z^{n,k} - T(z^{n,k})||_P^2                                */
  double  omega;                /* primal weight in force at iteration t                      */
  int32_t restart;              /* 1 if z^{n+1,0} = T(z^{n,k}) follows                         */
  int32_t retries;              /* adaptive step: rejected steps before this iteration's      */
  int64_t active;               /* check iterations: columns with x~ on a bound (the active
                                   set of Section 4's partition as the iterates see it); else -1 */
  int64_t changed;              /* check iterations: columns whose on-bound status changed since
                                   the previous recorded check; else -1 (also -1 for checks run
                                   by the mixed-precision restart kernels)                     */
} rhpdhg_trace_rec;

/* Fills *p with the defaults listed above.  Returns RHPDHG_OK, or RHPDHG_ERR_INVALID_ARG if
 * p is NULL. */
int rhpdhg_params_default(rhpdhg_params *p);

/* Validates and copies the LP to the current device, builds the transposed matrix, applies
 * Ruiz and Pock-Chambolle scaling (Section 7, "preprocessing"), estimates sigma_max(K^) by power
 * iteration and sets the step size and primal weight.  `cuda_stream` is a cudaStream_t of the
 * current device (NULL = the legacy default stream); all device work of the handle is ordered on
 * it.  On success *out holds a new handle (free with rhpdhg_free).  On failure *out is NULL and
 * rhpdhg_last_error(NULL) describes the error. */
int rhpdhg_create(const rhpdhg_problem *lp, const rhpdhg_params *params, void *cuda_stream,
                  rhpdhg_handle **out);

/* Runs Algorithm 1 or 2 (params.algorithm) from the initial point until a status is reached.
 * blocking = 1 returns when the solve has finished; blocking = 0 returns at once and a host
 * thread owned by the handle drives the device (poll reports completion).  Calling solve on a
 * handle whose solve is running returns RHPDHG_ERR_STATE; calling it again after completion
 * restarts from the initial point. */
int rhpdhg_solve(rhpdhg_handle *h, int blocking);

/* Non-blocking.  Returns RHPDHG_BUSY while the solve runs.  When done, fills *r (statistics,
 * and copies of x, y, cert_x, cert_y into the caller's non-NULL arrays of kind r->out_memory)
 * and returns RHPDHG_OK. */
int rhpdhg_poll(rhpdhg_handle *h, rhpdhg_result *r);

/* Requests cancellation of a running solve (status CANCELLED once the in-flight graph
 * launches drain).  No effect on an idle handle. */
int rhpdhg_cancel(rhpdhg_handle *h);

/* Waits for any running solve, releases all device and host resources.  NULL-safe. */
void rhpdhg_free(rhpdhg_handle *h);

/* Message of the last error on h (or of the last failed create when h is NULL).  The string is
 * owned by the library and valid until the next call on the same handle. */
const char *rhpdhg_last_error(const rhpdhg_handle *h);

/* ---- inspection (tests and tools) -------------------------------------------------------
 * All copies below go to host memory and synchronise the handle's stream; they return
 * RHPDHG_ERR_STATE while a solve is running. */

/* Copies the scaled-space state: which = 0 current iterate z^{n,k} (x, y);
 * 1 = last PDHG point T(z) (x~, y~); 2 = anchor z^{n,0}.  x holds n, y holds m doubles (either
 * may be NULL).  In FP32 precision the iterate is widened to double. */
int rhpdhg_get_state(const rhpdhg_handle *h, int which, double *x, double *y);

/* Copies the diagonal scalings D (m) and E (n) with K^ = D K E, and the step data. Any pointer
 * may be NULL. */
int rhpdhg_get_scaling(const rhpdhg_handle *h, double *D, double *E, double *eta,
                       double *omega0, double *sigma_max);

/* Copies up to `capacity` trace records (params.trace = 1) of the last solve; *count receives
 * the number recorded (min(iterations, trace_capacity)). */
int rhpdhg_get_trace(const rhpdhg_handle *h, rhpdhg_trace_rec *recs, int64_t capacity,
                     int64_t *count);

/* Launch geometry and walk layout chosen at create (for inspection and tests); out receives
 * RHPDHG_LAYOUT_FIELDS values: CTAs of the row kernels and of the column kernels; short tiles
 * walked per work item on K^ and on K^T (1, 2 or 4); long rows of K^ and of K^T; their chunks on
 * K^ and on K^T; the staging stride (entries per warp) of K^ and of K^T; the walk of the
 * ordinary mixed-precision kernels on K^ and on K^T (0 = one tile per item, 1 = one tile per
 * item with twice the loads in flight per staging round, 2 = groups of tiles per item; 0 for
 * FP64 handles); warps per CTA of the row kernels and of the column kernels; the autotuner's
 * outcome (0 = the fixed rule, 1 = timed at create, 2 = taken from the cache), and the time of
 * one iteration (row plus column stage, median, nanoseconds) with the rule's geometry and with
 * the chosen one (0 when not tuned); whether the FP64 walks of K^ and of K^T sum a tile's longest
 * rows warp-wide (1) or every row in one lane (0), decided at create from the row lengths.
 * capacity: entries available at out.  Returns RHPDHG_OK, or RHPDHG_ERR_INVALID_ARG for a NULL
 * handle or out, or capacity < RHPDHG_LAYOUT_FIELDS. */
#define RHPDHG_LAYOUT_FIELDS 19
int rhpdhg_get_layout(const rhpdhg_handle *h, int64_t *out, int32_t capacity);

/* Handles take their device buffers from a process-wide cache of buffers freed by earlier
 * handles (same device, same size; at most 4 GiB kept), so that creating and freeing handles of
 * the same sizes costs no device allocation after the first time.  This frees every cached
 * buffer (for instance before a device reset, or to give the memory back) and returns the bytes
 * freed.  Handles alive at the time are not affected. */
int64_t rhpdhg_release_cached_memory(void);

/* Plan of the tiled split-CSR layout that rhpdhg_create builds for an operator side (K^ or K^T)
 * with nrows rows and row pointers row_ptr (host memory, nrows + 1 entries, row_ptr[0] = 0); no
 * device is used.  out receives RHPDHG_PLAN_FIELDS values: 32-row tiles; short tiles per work
 * item (1, 2 or 4); long rows; long-row chunks; staging stride (entries per warp); padded
 * short-array entries; padded long-array entries; 1 if the FP64 walks sum each tile's longest
 * rows warp-wide (when that saves at least 15% of the FP64 adds of the row sums by the tile cost
 * model: lane-per-row sums cost the longest short row rounded up to 4, a threshold c of 8, 16 or
 * 32 costs c plus ceil(len / 32) + 5 per longer row), else 0.  capacity: entries available at out.
 * Returns RHPDHG_OK, or RHPDHG_ERR_INVALID_ARG for a NULL pointer, nrows < 0, row pointers that
 * do not start at 0 or decrease, offsets beyond int32, or capacity < RHPDHG_PLAN_FIELDS. */
#define RHPDHG_PLAN_FIELDS 8
int rhpdhg_plan_layout(const int64_t *row_ptr, int32_t nrows, int64_t *out, int32_t capacity);

/* With params.profile = 1: average device time (ms) per launch of the row-side kernel
 * (K x~ product + dual step) and of the column-side kernel (K^T y~ product + primal step) over
 * the last solve, their launch counts, and the algorithmic bytes one launch of each moves. */
int rhpdhg_kernel_times(const rhpdhg_handle *h, double *ms_row, double *ms_col,
                        int64_t *launches_row, int64_t *launches_col, double *bytes_row,
                        double *bytes_col);

/* Relative KKT error of an arbitrary point, the solver's termination measure (Section 7,
 * "Termination criteria"; l2 form, see rhpdhg_params.eps_rel_kkt): for the LP `lp`, whose arrays
 * must be in device memory (lp->memory = RHPDHG_MEM_DEVICE), and the unscaled point x (n
 * doubles) and y (m doubles) in device memory, writes to the host array out:
 *     out[0] = rel_p, out[1] = rel_d, out[2] = rel_gap, out[3] = primal_obj, out[4] = dual_obj.
 * Only the CSR of K is needed: K^T y is accumulated with atomic FP64 adds, so the last digits
 * may differ from run to run.  The CSR is not validated beforehand: a row whose offsets leave
 * [0, nnz] or decrease, and an entry whose column leaves [0, n), are skipped on the device and
 * the call then returns RHPDHG_ERR_INVALID_ARG.  Work is ordered on `cuda_stream` (NULL = legacy
 * default stream) and the call synchronises it, so it must not be issued on a stream that is
 * being captured into a graph.  Scratch (n + 8200 doubles) is allocated with cudaMalloc and
 * freed before returning.  Errors: RHPDHG_ERR_INVALID_ARG for host-memory, incomplete or
 * out-of-range input, RHPDHG_ERR_OOM / RHPDHG_ERR_CUDA on CUDA failures; each sets the message
 * of rhpdhg_last_error(NULL). */
int rhpdhg_kkt_eval(const rhpdhg_problem *lp, const double *x, const double *y,
                    void *cuda_stream, double *out);

/* Same evaluation as rhpdhg_kkt_eval, for callers that may not allocate device memory (for
 * instance code inside a framework that owns all device memory through its own pool, or a
 * latency-critical loop that must not take cudaMalloc's device-wide synchronisation).  The
 * paper has no counterpart to this call; it exists for those callers only.
 *   - Allocates nothing: no cudaMalloc, cudaFree or allocating library routine.  Its scratch is a
 *     fixed array of (2^20 + 8200) doubles (about 8.1 MiB) at file scope in the library, held by
 *     every GPU that loads the library until the process exits.
 *   - Size limit: n <= 1,048,576 (2^20).  Larger problems return RHPDHG_ERR_INVALID_ARG with a
 *     message in rhpdhg_last_error(NULL); use rhpdhg_kkt_eval for them.
 *   - The first call on each device looks up the array's device address (with that device
 *     current) and keeps it.  Every call copies its results to the host and synchronises the
 *     stream, so no call may be issued on a stream that is being captured into a graph.
 *   - All calls share the one array, and it keeps the previous call's contents (the call clears
 *     what has to start at zero).  Calls that overlap on the GPU, on any stream or from any host
 *     thread, race on the array and give wrong results: order them.
 * Arguments, results and other errors are those of rhpdhg_kkt_eval. */
int rhpdhg_kkt_eval_noalloc(const rhpdhg_problem *lp, const double *x, const double *y,
                            void *cuda_stream, double *out);

/* ---- rate probes (roofline denominators) ------------------------------------------------
 * Measurements of the current device for the bounds the iteration kernels are compared with;
 * neither changes a device setting.  Each times its kernel with CUDA events on cuda_stream
 * (NULL = legacy default stream) after one untimed launch, reports the best launch, allocates
 * and frees its own buffers and synchronises the stream.  Errors: RHPDHG_ERR_INVALID_ARG for a
 * NULL output or a size out of range, RHPDHG_ERR_OOM / RHPDHG_ERR_CUDA on CUDA failures, each
 * with a message in rhpdhg_last_error(NULL). */

/* FP64 fused multiply-add rate in TFLOP/s (2 flops per FMA): every resident thread runs 8
 * independent FMA chains. */
int rhpdhg_probe_fp64_fma_rate(void *cuda_stream, double *tflops);

/* Read bandwidth in GB/s of a device buffer of `bytes` (1 MiB .. 4 GiB) read repeatedly with
 * 16-byte loads that bypass L1: a size well inside L2 (for instance 64 MiB of the 126 MB) gives
 * the L2 read bandwidth, a size well beyond it the DRAM read bandwidth. */
int rhpdhg_probe_l2_read_bandwidth(int64_t bytes, void *cuda_stream, double *gbs);

/* ---- batched solver ---------------------------------------------------------------------
 * Many small LPs advance together in one persistent launch, one CTA per LP (the CTA also runs
 * the LP's set-up: scaling, power iteration, primal weight).  Each LP's computation stays inside
 * its CTA, so its result does not depend on which other LPs share the launch.  The method and
 * its statuses are those of rhpdhg_solve, in FP64 or (per slot) mixed precision.  Slots are
 * described by a table in device memory, so one captured graph is replayed while LPs are added
 * and removed. */
typedef struct rhpdhg_batch rhpdhg_batch;

/* Creates a batch with max_slots slots and a device arena of arena_bytes for the LPs' data.
 * cuda_stream: stream of all work (NULL = a private stream). */
int rhpdhg_batch_create(int32_t max_slots, int64_t arena_bytes, void *cuda_stream,
                        rhpdhg_batch **out);

/* Copies an LP (host memory, validated and transposed on the host) into a free slot; its set-up
 * runs in the next step.  params: as for rhpdhg_create (NULL = defaults; the constant step only).
 * precision 1 runs the slot's ordinary iterations with FP32 matrix values and FP32 offsets from
 * FP64 anchors, and its restarts, restart points and checks in FP64, like rhpdhg_solve (the
 * restart-norm sums are FP32 within each warp and FP64 across warps; a near-certificate at a
 * restart point moves the slot to FP64 for the rest of its solve).
 * Returns RHPDHG_BUSY when no slot is free and RHPDHG_ERR_OOM when the arena lacks
 * rhpdhg_batch_bytes_needed(lp, precision) contiguous bytes. */
int rhpdhg_batch_add(rhpdhg_batch *b, const rhpdhg_problem *lp, const rhpdhg_params *params,
                     int32_t *slot);

/* One launch: every active slot advances by up to iters PDHG evaluations (or runs its set-up and
 * then iterates).  Synchronises the batch stream and refreshes every slot's status. */
int rhpdhg_batch_step(rhpdhg_batch *b, int32_t iters);

/* RHPDHG_BUSY while the slot's LP runs; then fills *r like rhpdhg_poll (solve_seconds = 0). */
int rhpdhg_batch_poll(rhpdhg_batch *b, int32_t slot, rhpdhg_result *r);

/* Frees a slot (finished or not) and its arena region. */
int rhpdhg_batch_remove(rhpdhg_batch *b, int32_t slot);

/* Status of a slot after the last step (RHPDHG_STATUS_*), or -1 for an empty slot. */
int rhpdhg_batch_slot_status(const rhpdhg_batch *b, int32_t slot);

/* Free arena bytes (sum of free regions), and the bytes one LP needs in a slot of the given
 * precision (0 or 1; -1 for a NULL lp or another precision). */
int64_t rhpdhg_batch_free_bytes(const rhpdhg_batch *b);
int64_t rhpdhg_batch_bytes_needed(const rhpdhg_problem *lp, int32_t precision);

/* Kernel launches issued by the batch so far (steps and result extractions). */
int64_t rhpdhg_batch_launch_count(const rhpdhg_batch *b);

void rhpdhg_batch_free(rhpdhg_batch *b);

/* ---- serving: continuous batching under a device-memory budget ---------------------------
 * A worker thread admits submitted LPs first-come first-served while the budget allows (a
 * later request may pass one that does not fit yet).  LPs with at most small_nnz nonzeros
 * (and the constant step) become slots of an internal batched solver, in the precision the
 * request asks for (its arena, budget_bytes / 4 at most, counts against the budget); the others
 * get their own single-LP handle, solved on its own
 * stream concurrently with the batch.  Memory is released as each request finishes, and waiting
 * requests are admitted in the next turn.  Results are kept until polled. */
typedef struct rhpdhg_server rhpdhg_server;

/* budget_bytes: device memory the server may use; small_nnz: largest LP sent to the batched
 * solver; max_slots: batched slots; iters_per_step: iterations per batched launch. */
int rhpdhg_server_create(int64_t budget_bytes, int64_t small_nnz, int32_t max_slots,
                         int32_t iters_per_step, rhpdhg_server **out);

/* Copies the LP (host memory) and params (NULL = defaults) and queues it; *ticket identifies
 * it.  The submitter may free its arrays on return. */
int rhpdhg_server_submit(rhpdhg_server *s, const rhpdhg_problem *lp, const rhpdhg_params *params,
                         int64_t *ticket);

/* RHPDHG_BUSY until the request is finished; then fills *r (host arrays given in r, as in
 * rhpdhg_poll; solve_seconds = time from admission to completion), sets *latency_s (may be
 * NULL) to the time from submission to completion, and forgets the request. */
int rhpdhg_server_poll(rhpdhg_server *s, int64_t ticket, rhpdhg_result *r, double *latency_s);

/* Cancels a request (pending or running); its poll then reports RHPDHG_STATUS_CANCELLED. */
int rhpdhg_server_cancel(rhpdhg_server *s, int64_t ticket);

/* out[10]: pending, running batched, running single, completed, bytes in use, peak bytes in
 * use, budget, batched launches, admitted batched, admitted single. */
int rhpdhg_server_stats(rhpdhg_server *s, int64_t *out);

/* Stops the worker (running solves are abandoned) and frees everything.  NULL-safe. */
void rhpdhg_server_free(rhpdhg_server *s);

/* Number of CUDA kernels of this library the handle has launched so far (create and every
 * solve; a replay of a captured graph counts each kernel node it runs).  Kernels of the CUB
 * library used for the transpose during create are not counted.  Returns -1 for NULL. */
int64_t rhpdhg_launch_count(const rhpdhg_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* RHPDHG_H */
