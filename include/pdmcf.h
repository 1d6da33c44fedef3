/*
 * pdmcf.h — C ABI of the GB300 (sm_103a) PDMCF solver library (libpdmcf.so).
 *
 * Solves the all-pairs multicommodity network flow problem with destination-aggregated
 * flows (Zhang & Boyd, "Solving Large Multicommodity Network Flow Problems on GPUs",
 * Sec. 1.1, Eq. (e-prob)):
 *
 *     maximize   U(T) = sum_{i != j} u_ij(T_ij)
 *     subject to F >= 0,  F^T 1 <= c,  T + F A^T = 0
 *
 * by the PDMCF method (Algorithm 2.1): PDHG with over-relaxation (Eq. e-pdhg-step) on the
 * reduced Lagrangian (Eq. e-L), capped-simplex projection per edge (Sec. 2.3), entrywise
 * utility proxes (Sec. 2.3), adaptive primal weight (Eq. e-primal_weight) and the step
 * bound eta = 1/sqrt(2 d_max) (Eq. e-eta).
 *
 * Conventions (Sec. 1.1):
 *   - nodes are 0..n-1, edge l goes from tail[l] to head[l]; the incidence matrix has
 *     A[head[l], l] = +1, A[tail[l], l] = -1;
 *   - T[i*n + j] (row-major) is the traffic from source j to destination i; the diagonal
 *     holds T_ii = -sum_{j != i} T_ij, so T 1 = 0;
 *   - F[i*m + l] (row-major) is the flow on edge l destined to node i;
 *   - w[i*n + j] weights the utility of traffic j -> i; the diagonal is ignored.
 *
 * All functions return an int status (MCF_OK = 0 or a negative MCF_ERR_* code, or
 * MCF_PENDING). On error, mcf_last_error() returns a message for the calling thread.
 * Every function is safe to call from any thread; one problem handle must not be used by
 * two calls at the same time (mcf_submit'ed work counts as a use until it completes).
 * All solves run on the GPU; the library has no CPU fallback and fails with
 * MCF_ERR_CUDA when no usable CUDA device is present.
 */
#ifndef PDMCF_H
#define PDMCF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define MCF_OK                 0
#define MCF_PENDING            1   /* mcf_poll: the ticket has not finished yet        */
#define MCF_ERR_INVALID       -1   /* bad argument (sizes, ids, c <= 0, w <= 0, gamma) */
#define MCF_ERR_NOT_CONNECTED -2   /* network is not strongly connected (Sec. 1.1)     */
#define MCF_ERR_OOM           -3   /* device allocation failed                         */
#define MCF_ERR_CUDA          -4   /* CUDA runtime error / no device                   */
#define MCF_ERR_NUMERIC       -5   /* NaN or Inf in the iterates                       */
#define MCF_ERR_NOT_CONVERGED -6   /* max_iters reached; results are still filled      */
#define MCF_ERR_TIMEOUT       -7   /* mcf_wait timed out                               */
#define MCF_ERR_BUSY          -8   /* queue full, or the problem has an outstanding ticket */
#define MCF_ERR_OOM_BUDGET    -9   /* instance does not fit the serving HBM budget     */
#define MCF_ERR_CANCELLED    -10   /* ticket cancelled before it completed             */

/* ---------------------------------------------------------------- enums */
#define MCF_LOG 0          /* u(s) = w log s                     (Sec. 1.1) */
#define MCF_POW 1          /* u(s) = w s^gamma, gamma in (0, 1)  (Sec. 1.1) */

#define MCF_FP32   0       /* float iterates, float storage of F                       */
#define MCF_FP64   1       /* double iterates (small problems, exact parity checks)     */
#define MCF_BF16_F 2       /* float iterates, bfloat16 storage of F, float accumulation */

#define MCF_STOP_PAPER   0 /* stop when r^k < n m eps (Sec. 2.5, residual of Eq. e-res)   */
#define MCF_STOP_REL_KKT 1 /* stop when the relative KKT measure (see mcf_result) < eps  */
#define MCF_STOP_NONE    2 /* run exactly max_iters iterations                           */

typedef struct mcf_problem mcf_problem;   /* opaque */
typedef int64_t mcf_ticket;

/* ---------------------------------------------------------------- options */
typedef struct mcf_options {
  double  eps;               /* tolerance for the stop test (default 1e-4)                 */
  int     stop_mode;         /* MCF_STOP_* (default MCF_STOP_REL_KKT)                       */
  int64_t max_iters;         /* iteration cap (default 100000)                              */
  double  rho;               /* over-relaxation, Sec. 2.2 (default 1.9)                     */
  double  theta;             /* primal weight smoothing, Eq. e-primal_weight (default 0.5)  */
  int     k_adapt;           /* primal weight period, Sec. 2.4 (default 100)                */
  double  tau;               /* primal weight threshold on Delta_F, Delta_Y (default 1e-5)  */
  int64_t omega_freeze_iter; /* stop adapting omega from this iteration on; -1 = never      */
  int     k_check;           /* stop test every k_check iterations (default 50)             */
  int     precision;         /* MCF_FP32 | MCF_FP64 | MCF_BF16_F (default MCF_FP32)         */
  int     warm_start;        /* 1: start from the problem's resident (F, Y, omega)          */
  int     polish_iters;      /* MCF_BF16_F: extra FP32 iterations after convergence         */
  int     use_graphs;        /* capture each k_check-iteration chunk in a CUDA graph (1)    */
  int     device;            /* CUDA device ordinal (default 0)                             */
  void*   cuda_stream;       /* cudaStream_t to run on; NULL = the library's own stream     */
  double  omega0;            /* initial primal weight for cold starts (default 1.0)         */
  int     stall_checks;      /* stop when the relative KKT measure has not improved by 5 %
                                over this many consecutive checks while within 100x of eps
                                (FP32 iterates reach a rounding floor); the count restarts
                                when omega stops adapting; 0 = never. The result then has
                                stalled = 1 and status MCF_ERR_NOT_CONVERGED. Default 100   */
  int     compensated_duals; /* FP32/BF16 iterates: keep Y as an FP32 head plus a BF16 tail
                                so the dual update is not limited by FP32 spacing of large
                                duals (default 1; ignored for MCF_FP64)                     */
  int     autotune;          /* batched and served solves: pick each size class's launch
                                shape by timing candidates once per process on synthetic
                                instances of that size (default 1)                         */
  int     shape;             /* kernel launch shape index (-1 = automatic); see
                                mcf_shape_info. Lets tests and the tuner pick any shape
                                whose capacity covers the problem                          */
  double  adapt_guard;       /* g: stop adapting omega (keep it constant, Sec. 2.4) from
                                the iteration after a stop test where omega is more than a
                                factor g^2 away from its value at the first stop test with
                                a finite relative KKT measure, or, once that measure has
                                been below adapt_guard_below (the final phase), where omega
                                is more than a factor g away from its value when that phase
                                began or a finite measure exceeds g x the smallest one of
                                the solve. 0 = adapt throughout (default 10). The result
                                reports the iteration in omega_frozen_at.                  */
  double  adapt_guard_below; /* start of the final phase for adapt_guard (default 1e-2)   */
  const char* check_log;     /* path of a file to which mcf_solve and mcf_solve_timed append
                                one JSON line per stop test (every k_check iterations): k,
                                omega, r/(n m), rel_kkt and its three parts, U, D, the
                                fraction of nonpositive off-diagonal T, whether omega still
                                adapts, the precision (the convergence diagnostics of
                                Sec. 3.1); NULL = none (default). Non-finite values are
                                written as null. Not used by batched or served solves      */
} mcf_options;

/* ---------------------------------------------------------------- results */
typedef struct mcf_result {
  /* caller-owned output buffers (host memory), each optional (NULL = not wanted) */
  double* T;           /* n*n, T[i*n+j]: traffic j -> i of the returned flow         */
  double* F;           /* n*m, F[i*m+l]: the returned (projected) flow  F^{k-1/2}    */
  double* Y;           /* n*n, Y[i*n+j]: the dual prox output Y^k                     */
  /* scalars (always filled) */
  int64_t iters;       /* PDHG iterations performed                                   */
  int     status;      /* MCF_OK, MCF_ERR_NOT_CONVERGED, MCF_ERR_NUMERIC, ...         */
  int     feasible;    /* 1 if every off-diagonal T_ij > 0 (Sec. 1.1 domain)          */
  double  utility;     /* U(T), FP64 reduction (-inf if not feasible)                 */
  double  dual_bound;  /* D(Y) >= U*: (-U)^*(Y) + sum_l c_l max(0, max_i (Y A)_il)     */
  double  r;           /* residual r^k of Eq. (e-res) (inf if not feasible)            */
  double  r_over_nm;   /* r / (n m), the paper's normalised residual                   */
  double  rel_gap;     /* (D - U) / (1 + |U| + |D|)                                    */
  double  rel_cons;    /* ||T(Y) - T||_F / (1 + ||T||_F), T(Y) = (u')^{-1}(-Y), off-diag */
  double  rel_stat;    /* sqrt(r) / (1 + ||G||_F), G = U'A (Sec. 1.2)                  */
  double  rel_kkt;     /* max(rel_gap, rel_cons, rel_stat)                             */
  double  nonpos_frac; /* fraction of off-diagonal T_ij <= 0 (Sec. 3.1 diagnostic)      */
  double  omega;       /* final primal weight                                          */
  int     stalled;     /* 1 if the stall rule (mcf_options.stall_checks) ended the solve */
  double  delta_f;     /* Delta_F of the last iteration (Eq. e-primal_weight)           */
  double  delta_y;     /* Delta_Y of the last iteration                                 */
  int64_t omega_frozen_at; /* iteration from which omega stayed constant (-1: never)     */
  double  seconds;     /* wall time of the call                                        */
} mcf_result;

/* ---------------------------------------------------------------- problem lifecycle */

/* Create a problem from the data of Eq. (e-prob) (Sec. 1.1).
 *   n, m          node and edge counts (n >= 2, m >= 1)
 *   tail, head    m edge endpoints, 0 <= id < n, tail != head, no duplicate pairs; the
 *                 network must be strongly connected (Sec. 1.1), else MCF_ERR_NOT_CONNECTED
 *   cap           m capacities c_l > 0
 *   utility_kind  MCF_LOG or MCF_POW
 *   w             n*n weights, w[i*n+j] > 0 for i != j (diagonal ignored)
 *   gamma         MCF_POW only: NULL with gamma_len = 0 is invalid for MCF_POW; gamma_len
 *                 = 1 (one exponent) or n*n (per pair, row-major like w); each in (0, 1)
 *   out           receives the handle
 * All arrays are host memory, copied; the caller keeps ownership. Device memory is
 * allocated at the first solve, on the device named in its options. */
int mcf_create_problem(int32_t n, int32_t m, const int32_t* tail, const int32_t* head,
                       const double* cap, int utility_kind, const double* w,
                       const double* gamma, int64_t gamma_len, mcf_problem** out);

/* Replace the capacities (m values > 0). The resident iterate (F, Y, omega) is kept, so
 * a following solve with warm_start = 1 re-solves from it (Sec. 3.1, warm start). */
int mcf_update_capacities(mcf_problem* p, const double* cap);

/* Replace the weights (n*n host values, > 0 off the diagonal); resident state kept. */
int mcf_update_weights(mcf_problem* p, const double* w);

/* Free the problem and its device memory. Must not be called while a ticket on it is
 * pending. NULL is accepted. The device memory goes back to the library's stream-ordered
 * pool for that device, which keeps up to 32 GB of freed memory for the next problem's
 * state (and gives cached memory back when an allocation would otherwise fail). */
int mcf_destroy_problem(mcf_problem* p);

/* Size queries. */
int mcf_problem_size(const mcf_problem* p, int32_t* n, int32_t* m);

/* The library's internal node numbering. Relabelling nodes leaves the problem of Sec. 1.1
 * unchanged. At creation the library renumbers the nodes in reverse Cuthill-McKee order
 * when that shortens the mean edge span |tail - head| at least 4x, which makes the
 * per-edge dual-row gathers local in memory. All inputs and outputs stay in the caller's
 * numbering.
 *   node_of  NULL, or n int32 (host): node_of[caller node] = internal node
 * Returns 1 if the nodes were renumbered, 0 if the internal numbering is the caller's
 * (node_of is then the identity), or a negative error code. */
int mcf_problem_node_order(const mcf_problem* p, int32_t* node_of);

/* The library's internal edge order: edges sorted by head (internal numbering), so each
 * node's in-edges are one contiguous block of rows of the edge-major F.
 *   edge_of  m int32 (host): edge_of[internal edge e] = the caller's edge index
 * It is also the row order of F in a file written by mcf_save_state. Returns MCF_OK. */
int mcf_problem_edge_order(const mcf_problem* p, int32_t* edge_of);

/* Device bytes one solve of this problem needs at the given precision. */
int64_t mcf_problem_device_bytes(const mcf_problem* p, int precision);

/* ---------------------------------------------------------------- solving */

/* Fill *o with the paper's defaults (Sec. 2.2, 2.4, 2.5) and the library defaults above. */
void mcf_options_default(mcf_options* o);

/* Run Algorithm 2.1 on the GPU until the stop test passes or max_iters is reached
 * (synchronous). Cold start: F^{-1/2} = 0, Y^0 = I - 1 1^T, omega^0 = omega0 (Sec. 2.5);
 * warm_start = 1 continues from the problem's resident iterate. Fills *res (scalars and
 * any non-NULL output buffers). Returns MCF_OK, MCF_ERR_NOT_CONVERGED (results filled),
 * MCF_ERR_NUMERIC, MCF_ERR_OOM, MCF_ERR_CUDA or MCF_ERR_INVALID. */
int mcf_solve(mcf_problem* p, const mcf_options* opts, mcf_result* res);

/* Solve `count` independent problems together on one GPU (FP32 iterates only): each PDHG
 * phase is one launch per launch-shape class for all resident problems, every problem keeps
 * its own step sizes, iteration count and stop test on the device, and its reductions are
 * summed per edge and per node in a fixed order, so a problem's iterates are identical
 * whether it is solved alone or in any batch. opts applies to every problem (warm_start = 1
 * continues each problem's resident iterate). results[i] is filled as by mcf_solve for
 * problems[i], including any output buffers it points to. The problems must be distinct
 * and not in use by other calls. Returns MCF_OK if every problem met its stop rule, else
 * the first other status (results are still filled). */
int mcf_solve_batch(mcf_problem** problems, int count, const mcf_options* opts,
                    mcf_result* results);

/* Asynchronous solve: enqueue and return a ticket at once. The serving scheduler admits
 * the request when its device footprint fits the HBM budget (mcf_serving_config) and
 * advances it batched with the other resident requests. The options are copied; the
 * problem must stay alive until the ticket is collected.
 * A problem has at most one outstanding ticket, from mcf_submit until the ticket is
 * collected: by the mcf_poll or mcf_wait that reports its final status, or by mcf_cancel
 * of a finished ticket. Its outputs are read from the problem's device state at
 * collection, so until then mcf_submit, mcf_solve, mcf_solve_batch, mcf_autotune,
 * mcf_update_capacities, mcf_update_weights and mcf_destroy_problem on that problem return
 * MCF_ERR_BUSY. Also MCF_ERR_BUSY when the queue is full; MCF_ERR_OOM_BUDGET when the
 * request's footprint alone exceeds the budget. */
int mcf_submit(mcf_problem* p, const mcf_options* opts, mcf_ticket* ticket);

/* Non-blocking: *status receives MCF_PENDING until the ticket finishes, then its final
 * status, and *res (if not NULL) is filled as by mcf_solve. The first poll that reports
 * the final status collects the ticket (its id is then unknown) and frees the problem for
 * new work. */
int mcf_poll(mcf_ticket ticket, int* status, mcf_result* res);

/* Blocking form of mcf_poll with a timeout in milliseconds (< 0: no limit). Returns
 * MCF_ERR_TIMEOUT if the ticket is still pending when the limit passes. */
int mcf_wait(mcf_ticket ticket, int64_t timeout_ms, int* status, mcf_result* res);

/* Cancel a ticket. Queued: removed at once. Running in the batched engine: it leaves its
 * slot at the next chunk boundary (every 10 iterations), keeping the iterate reached as the
 * problem's warm state. Running one at a time (MCF_FP64, MCF_BF16_F or a forced shape):
 * it runs to its stop rule. In each case the next poll reports MCF_ERR_CANCELLED and
 * collects it. Finished but not collected: its result is discarded and the ticket is
 * collected. */
int mcf_cancel(mcf_ticket ticket);

/* Serving configuration: HBM budget for admitted requests (bytes, > 0) and the maximum
 * number of requests resident at once (>= 0; 0 pauses admission: requests queue but none
 * starts). Defaults: 120 GB, 256. */
int mcf_serving_config(int64_t hbm_budget_bytes, int max_resident);

/* Stop the serving threads. Every ticket not finished ends with MCF_ERR_CANCELLED: queued
 * ones at once, batched running ones after the chunk in progress (their problems keep
 * the iterate reached), a running one-at-a-time solve when it returns. Returns when both
 * threads have exited; their tickets are still collected by mcf_poll / mcf_wait. A later
 * mcf_submit starts the threads again. Library service; the paper has no counterpart. */
int mcf_serving_shutdown(void);

/* Per-kernel device times of a timed solve (CUDA events recorded on the solve stream
 * between consecutive kernels). Index 0 edge phase, 1 node phase, 2 residual check,
 * 3 scalar tail. */
typedef struct mcf_kernel_times {
  double  ms[4];         /* summed device time per kernel kind                        */
  int64_t launches[4];   /* launches per kernel kind                                  */
  double  ms_total;      /* first to last event of the iteration launches             */
  int     shape;         /* launch shape the solve used (an mcf_shape_info index)     */
} mcf_kernel_times;

/* As mcf_solve, but launches every kernel individually (no CUDA graphs) with a CUDA event
 * before and after it on the solve stream, and fills *kt. For measurement. */
int mcf_solve_timed(mcf_problem* p, const mcf_options* opts, mcf_result* res,
                    mcf_kernel_times* kt);

/* ---------------------------------------------------------------- operators on device arrays */

/* The projection Pi onto the feasible flow set of Sec. 2.3, one column at a time: for each
 * of the m columns q_l (row l of Qt), Ft row l = (q_l - mu_l 1)_+ where mu_l = 0 if
 * sum_i (q_il)_+ <= cap_l, else the unique mu_l > 0 with sum_i (q_il - mu_l)_+ = cap_l
 * (the value the sorted scan of Sec. 2.6 gives).
 *   n      column length (number of destinations), 1 <= n <= 32768
 *   m      number of columns (>= 0)
 *   ld     row stride of Qt and Ft in floats: ld >= n, ld % 4 == 0
 *   Qt     device, m x ld floats, 16-byte aligned; entries n..ld-1 of each row are ignored
 *   cap    device, m capacities > 0
 *   Ft     device, m x ld floats, 16-byte aligned; entries n..ld-1 are written as 0. Ft may
 *          equal Qt (in place)
 *   mu     device, m floats: on entry a starting guess (0 = none; any value >= 0 is valid),
 *          on exit the multipliers mu_l
 *   dist2  host, may be NULL: receives sum_l ||Ft_l - q_l||^2, an FP64 reduction in a fixed
 *          order (independent of the launch grid)
 *   stream cudaStream_t (NULL = legacy default stream), on the calling thread's current device
 * Allocates m+1 doubles of device scratch for the call and synchronizes the stream before
 * returning. Errors: MCF_ERR_INVALID (sizes, NULL or misaligned pointers), MCF_ERR_OOM,
 * MCF_ERR_CUDA. */
int mcf_project_capped_simplex(int32_t n, int32_t m, int32_t ld, const float* Qt,
                               const float* cap, float* Ft, float* mu, double* dist2,
                               void* stream);

/* The same projection for callers that cannot allocate device memory: processes whose
 * device memory belongs to their own pool or to a framework allocator that must see every
 * allocation, and loops that must never enter the allocator (a cudaMalloc can synchronize
 * the device and take milliseconds). The paper has no counterpart; this is a library
 * service. Arguments and results are those of mcf_project_capped_simplex, except:
 *   - no device memory is allocated or freed: the scratch (m + 1 doubles) is a fixed array in
 *     the library image, present on every GPU that loads the library until the process
 *     exits; m is limited to 262144 columns (MCF_ERR_INVALID beyond, nothing launched);
 *   - the first call on each device looks up that array's device address (and may load
 *     the library's device code); make that first call before any stream capture. The
 *     address is looked up again when the device's context has changed (for instance after
 *     a cudaDeviceReset by the application);
 *   - the call returns without synchronizing when dist2 is NULL (the work is queued on
 *     stream); with dist2 it waits for the result;
 *   - all calls share the one array: calls whose work overlaps on the GPU (different
 *     streams or host threads without ordering) race and give undefined results. Each call
 *     writes every scratch entry it reads, so nothing needs clearing between calls. */
int mcf_project_capped_simplex_noalloc(int32_t n, int32_t m, int32_t ld, const float* Qt,
                                       const float* cap, float* Ft, float* mu, double* dist2,
                                       void* stream);

/* Time every launch shape that covers this problem (register shapes up to 4x the smallest
 * sufficient capacity, and kinds 1 and 2 when opts->precision is not MCF_FP64) with
 * 3 + 10 iterations each, and return the fastest in *best_shape (for mcf_options.shape) and
 * its time per iteration in *ms_per_iter (may be NULL). Uses the problem's device state; the
 * next solve of the problem starts cold. */
int mcf_autotune(mcf_problem* p, const mcf_options* opts, int* best_shape, double* ms_per_iter);

/* Launch shape table: shape s gives `group` threads per edge/node, each holding `vpt`
 * chunks of the edge/node vector: for kind 0 a chunk is 16 bytes of F (4 FP32, 2 FP64 or
 * 8 BF16 entries), for kinds 1 and 2 it is 4 entries whatever the storage type; a shape
 * covers a problem when group*vpt chunks hold n rounded up to 8 entries.
 * kind[s]: 0 register shapes (grid-stride over edges); 1 bulk-copy pipelined edge phase
 * (cp.async.bulk into two shared-memory stages, one CTA per SM over head-aligned edge
 * ranges); 2 register edge phase over head-aligned edge ranges with per-head in-sums in
 * shared memory. Kinds 1 and 2 hand the in-sums to the node phase, need FP32 iterates, and
 * kind 2 is the automatic choice for rows of 8 KB or more. Returns the number of shapes;
 * fills the four arrays (each may be NULL) up to that count. */
int mcf_shape_info(int* group, int* vpt, int* block, int* kind);

/* ---------------------------------------------------------------- warm-state checkpoint */

/* Write the problem's resident warm state (Sec. 3.1 warm start: F^{k-1/2}, Y^k with its
 * compensated tail, the state F^{k-1/2} A^T of the relaxation identity, the projection
 * multipliers and omega) to a host file, in the library's internal layout. The problem must
 * have been solved (MCF_ERR_INVALID otherwise). Synchronizes the device. Errors:
 * MCF_ERR_INVALID (no state, file not writable), MCF_ERR_BUSY (outstanding ticket),
 * MCF_ERR_OOM, MCF_ERR_CUDA. */
int mcf_save_state(mcf_problem* p, const char* path);

/* Read a file written by mcf_save_state into the problem's device state on `device`
 * (allocating it if needed), so that the next solve with warm_start = 1 continues from it:
 * the result equals that of a warm solve of the problem the state was saved from, bit for
 * bit. The network (n, m, edges) must be the one the state was saved from; capacities and
 * weights are the problem's own. Errors: MCF_ERR_INVALID (unreadable or foreign file,
 * different network), MCF_ERR_BUSY, MCF_ERR_OOM, MCF_ERR_CUDA. The paper has no
 * counterpart for the file itself; it carries the warm start across processes. */
int mcf_load_state(mcf_problem* p, const char* path, int device);

/* ---------------------------------------------------------------- testing aids */

/* Exercise the bounded device-side waits: the next solve whose edge phase is the bulk-copy
 * pipelined kind (mcf_shape_info kind 1) arms the first shared-memory stage of its block 0
 * for copies that it never issues, in its first iteration. That stage's mbarrier wait then
 * gives up (2^22 polls or 2 s), the block drains its own copies (bounded the same way) and
 * returns, and the solve ends with MCF_ERR_CUDA ("a bounded device-side wait timed out");
 * no copy is left in flight and the context stays usable. The problem's iterate is then
 * invalid, so the next solve starts cold. The paper has no counterpart. Returns MCF_OK. */
int mcf_test_withhold_next_copy(void);

/* Message for the last error of the calling thread ("" if none). */
const char* mcf_last_error(void);

/* Library version string. */
const char* mcf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PDMCF_H */
