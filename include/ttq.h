/*
 * ttq.h - C ABI of the GB300 TT-cross quadrature library (libttq.so).
 *
 * The library computes tensor-product quadratures (Sec. 4.1, Eq. 5 of
 * Dolgov & Savostyanov, arXiv:1903.11554)
 *
 *     I = c * sum_{i_1..i_d} w_{1,i_1} ... w_{d,i_d} g(t_{1,i_1}, ..., t_{d,i_d})
 *
 * of the Ising-class integrands C_n, D_n, E_n (Sec. 5.1, Eqs. 9-11) by the
 * dimension-parallel greedy tensor-train cross (Alg. 6 with Alg. 2 on every
 * superblock at once), with the quadrature weights folded into the tensor
 * (Sec. 4.1) and the integral contracted from the TT cores and the inverse
 * cross matrices (Sec. 4.1, product of 2d-1 matrices).
 *
 * Conventions
 *  - All entry points return an int status: 0 = TTQ_OK, > 0 a warning,
 *    < 0 an error (see ttq_status).  No C++ exception crosses the ABI.
 *  - "host" pointers are read during the call only; the caller keeps
 *    ownership.  "device" pointers must stay valid while a plan uses them.
 *  - Streams are passed as void* (a cudaStream_t; NULL = legacy default).
 *  - All compute runs in the library's own CUDA kernels (sm_103a); there is
 *    no CPU fallback: without a usable GPU every entry point that computes
 *    returns TTQ_ERR_CUDA.
 *  - A plan is not thread-safe; use one plan per thread.
 */
#ifndef TTQ_H
#define TTQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Integrand families, Sec. 5.1 (Eqs. 9-11).  TEST is a separable tensor of
 * exact TT rank n (g = sum_{t=1}^n exp(-t * mean(x))), used to check the exact
 * recovery theorem (Thm. 2); it has no counterpart among the paper's integrals. */
typedef enum { TTQ_FAMILY_C = 0, TTQ_FAMILY_D = 1, TTQ_FAMILY_E = 2, TTQ_FAMILY_TEST = 3 } ttq_family;

/* Variables of the integral.
 *  TTQ_FORM_RN:   s in R^n, d = n modes; C_n = 4/n! int (sum 2cosh s_j)^-2,
 *                 D_n adds prod_{i<j} tanh^2((s_i - s_j)/2).  Nodes are s values.
 *  TTQ_FORM_CUBE: the paper's form on [0,1]^(n-1), d = n-1 modes x_2..x_n
 *                 (Eqs. 9-11), constant 2.  Nodes are x values in [0,1].     */
typedef enum { TTQ_FORM_RN = 0, TTQ_FORM_CUBE = 1 } ttq_form;

/* Arithmetic of the final contraction (Sec. 4.1): plain FP64, or double-double
 * node sums and chain products (compensated TwoSum / FMA-based TwoProd).  The
 * integrand, the QR of the cross matrices and the interface solves are FP64
 * in both modes.  In double-double mode the per-sweep values that drive the
 * stopping rule are FP64 contractions; the reported value (and value_lo) is
 * the double-double contraction of the final index sets. */
typedef enum { TTQ_PREC_FP64 = 0, TTQ_PREC_DD = 1 } ttq_precision;

typedef enum {
  TTQ_OK = 0,
  TTQ_WARN_NO_PIVOT = 1,      /* stopped: no interface accepted a pivot            */
  TTQ_WARN_RANK_CAP = 2,      /* stopped: every interface at the rank cap          */
  TTQ_WARN_MAX_SWEEPS = 3,    /* stopped: sweep limit reached before convergence   */
  TTQ_PENDING = 4,            /* serving: request not finished yet                 */
  TTQ_ERR_INVALID_ARG = -1,
  TTQ_ERR_NONFINITE = -2,     /* the integrand produced inf/nan                    */
  TTQ_ERR_SINGULAR = -3,      /* a cross matrix A(I<=k, I>k) became singular       */
  TTQ_ERR_WORKSPACE = -4,     /* workspace too small or misaligned                 */
  TTQ_ERR_CUDA = -5,          /* a CUDA call failed (message: ttq_last_error)      */
  TTQ_ERR_ADMISSION = -6,     /* serving: request larger than the memory budget    */
  TTQ_ERR_NOT_FOUND = -7,
  TTQ_ERR_TIMEOUT = -8        /* the persistent search gave up waiting (ttq_plan_set_wait_limit) */
} ttq_status;

#define TTQ_MAX_MODES 32      /* d <= 32 */
#define TTQ_MAX_RANK 128      /* rank cap <= 128 */
#define TTQ_MAX_NODES 2048    /* N_k <= 2048 */
#define TTQ_MAX_INIT_SAMPLES 1024
#define TTQ_MAX_PIVOTS 4      /* pivots an interface may add per sweep (npiv) */

/* The problem statement (Sec. 4.1: integrand, per-mode nodes and weights;
 * Alg. 6 inputs: rank cap and stopping tolerance). */
typedef struct ttq_problem {
  int32_t family;             /* ttq_family */
  int32_t form;               /* ttq_form */
  int32_t n;                  /* Ising index (TEST: number of separable terms) */
  int32_t d;                  /* number of modes: n (RN), n-1 (CUBE), any (TEST) */
  const int32_t *nodes_per_mode;  /* host [d], N_k in 2..TTQ_MAX_NODES */
  const double *nodes;        /* [sum N_k] node values, mode-major; host or device */
  const double *weights;      /* [sum N_k] quadrature weights, same layout */
  int32_t inputs_on_device;   /* 1: nodes/weights are device pointers */
  int32_t rank_cap;           /* 1..TTQ_MAX_RANK */
  double tol;                 /* stop when |I_s - I_{s-1}| <= tol |I_s| in conv_window sweeps in a row */
  double pivot_tol;           /* keep a pivot when |E*| > pivot_tol * max|core entry| */
  int32_t conv_window;        /* >= 1 */
  int32_t max_sweeps;         /* > 0 */
  uint64_t seed;              /* counter-based SplitMix64 key of the random samples */
  int32_t n_samples;          /* random samples per interface; 0 -> N_k + N_{k+1} */
  int32_t rook_max;           /* column/row rounds of rook pivoting, >= 1 */
  int32_t init_samples;       /* random points scanned for the initial multi-indices, 1..TTQ_MAX_INIT_SAMPLES */
  int32_t precision;          /* ttq_precision */
  int32_t r0;                 /* initial multi-indices (the rank of every interface before the first sweep),
                                 1..rank_cap and at most min(N_1, N_d, init_samples); 0 is taken as 1 */
  int32_t npiv;               /* pivots an interface may add per sweep, 0..TTQ_MAX_PIVOTS; 0 or 1: one, as
                                 Alg. 6.  More (a rank-adaptive variant): the npiv best random samples with
                                 distinct rows and columns start rook searches (Alg. 2) on the sweep's old
                                 residual (a search that meets an earlier one at the same step stops there:
                                 its end would be the earlier one's pivot), and greedy complete pivoting on
                                 the residual matrix of their rows and columns keeps the pairs whose Schur
                                 pivot passes the acceptance threshold, appended in that order.  Single
                                 plans of the staged search only (not batches, servers, the persistent or
                                 the sequential search). */
} ttq_problem;

typedef struct ttq_result {
  double value;               /* integral (family constant included) */
  double value_lo;            /* double-double tail (0 in FP64 mode) */
  double internal_conv;       /* last relative change |I_s - I_{s-1}| / |I_s| */
  int64_t n_eval;             /* integrand evaluations: core entries + search + initial scan */
  int32_t sweeps;             /* sweeps run (each with its own integral value) */
  int32_t max_rank;
  int32_t status;             /* ttq_status of the run */
  int32_t d;                  /* number of modes */
  int32_t ranks[TTQ_MAX_MODES + 1];   /* final TT ranks r_0 = 1, r_1 .. r_{d-1}, r_d = 1 (entries past d are 0) */
} ttq_result;

/* Per-interface outcome of one pivot search (Alg. 2 on superblock k).  The
 * argmax of every step treats candidates whose |E| lies within
 * 1e-12 * max + 1e-14 * max|core entry| of the maximum as tied and takes the
 * first in scan order (the paper does not define ties). */
typedef struct ttq_pivot {
  int32_t k;                  /* interface 1..d-1 */
  int32_t searched;           /* 0 if the interface was at the cap or stopped */
  int32_t row;                /* rho = alpha * N_k + i */
  int32_t col;                /* gamma = j * r_{k+1} + beta */
  double err;                 /* residual A - A~ at the pivot */
  int32_t accepted;
  int32_t rounds;             /* rook rounds run */
  int64_t evals;              /* integrand evaluations of this search */
} ttq_pivot;

typedef struct ttq_plan ttq_plan;

/* Device workspace (bytes, 256-byte aligned) a plan for this problem needs.
 * It holds the node tables, index sets, cores, QR factors and search state;
 * its size grows as sum_k cap^2 N_k. */
int ttq_workspace_bytes(const ttq_problem *p, size_t *bytes);

/* Create a plan over caller-owned device memory `workspace` (>= the size
 * above, 256-byte aligned).  Copies the problem's nodes/weights to the
 * workspace on `stream` (host->device when inputs_on_device == 0) and builds
 * the derived node tables.  The plan object itself lives in host memory. */
int ttq_plan_create(const ttq_problem *p, void *workspace, size_t bytes, void *stream, ttq_plan **out);
int ttq_plan_destroy(ttq_plan *plan);

/* Full run: initial index set, then sweeps until a stopping rule fires
 * (Alg. 6 repeated).  Blocks until the result is on the host.  On a stream
 * other than the legacy default stream, one sweep is captured once into a
 * CUDA graph and replayed; the contraction runs on a second stream of the
 * plan, beside the pivot search. */
int ttq_plan_run(ttq_plan *plan, ttq_result *out);

/* Asynchronous pair: ttq_plan_launch enqueues a whole run on the plan's
 * stream (one CUDA graph) followed by a copy of its final state into result
 * slot `slot` (0..63, pinned host memory owned by the plan) and returns at
 * once; ttq_plan_result waits for the stream and reads that slot.  Runs of
 * one plan execute in launch order; a slot is valid until it is launched
 * into again.  Without graphs (legacy default stream, or graphs switched off)
 * ttq_plan_launch runs synchronously. */
int ttq_plan_launch(ttq_plan *plan, int slot);
int ttq_plan_result(ttq_plan *plan, int slot, ttq_result *out);

/* --- the tensor train as a result ------------------------------------------
 * Alg. 6 returns the TT cross itself: the cores Y_k = A(I<=k-1, i_k, I>k)
 * (Eq. 3, weights folded, Sec. 4.1) and the nested index sets (Eq. 4) that
 * define them.  ttq_tt_export copies one instance's tensor train, for the
 * ranks of its last evaluated sweep, from the plan's workspace into a
 * caller-owned device buffer (>= ttq_tt_bytes, 256-byte aligned) and returns a
 * handle; it blocks until the copy is done, and the handle stays valid until
 * ttq_tt_free, whatever the plan does afterwards (the buffer stays the
 * caller's: free it after ttq_tt_free).  ttq_tt_get gives, for k = 1..d, the
 * shape and device pointers of core k (row-major r_{k-1} x N_k x r_k
 * doubles, family constant not included), of I<=k-1 (row-major
 * r_{k-1} x (k-1) int32 node indices of modes 1..k-1; NULL for k = 1) and of
 * I>k (row-major r_k x (d-k) node indices of modes k+1..d; NULL for k = d).
 * The integral is the product of 2d-1 matrices built from these (Sec. 4.1).
 * instance: 0 for a single plan, 0..count-1 for a batch. */
typedef struct ttq_tt ttq_tt;
int ttq_tt_bytes(ttq_plan *plan, int instance, size_t *bytes);
int ttq_tt_export(ttq_plan *plan, int instance, void *buffer, size_t bytes, ttq_tt **out);
int ttq_tt_get(const ttq_tt *tt, int k, int32_t *r_left, int32_t *n_k, int32_t *r_right, const double **core_dev,
               const int32_t **left_idx_dev, const int32_t **right_idx_dev);
int ttq_tt_ranks(const ttq_tt *tt, int32_t *d, int32_t *ranks /* [d+1] */);
int ttq_tt_free(ttq_tt *tt);

/* --- batches ---------------------------------------------------------------
 * Many integrals with uneven families, n, node counts and rank caps advance
 * together: every kernel launch of a sweep covers all instances (one
 * persistent-style launch per stage, instance = grid z), and the whole batch
 * runs as one CUDA graph whose WHILE loop continues while any instance is
 * running.  A batch is a ttq_plan with count instances (destroy with
 * ttq_plan_destroy); stage calls need count == 1.  Each instance's result is
 * exactly what a single plan gives for that problem. */
int ttq_batch_workspace_bytes(const ttq_problem *probs, int count, size_t *bytes);
int ttq_batch_create(const ttq_problem *probs, int count, void *workspace, size_t bytes, void *stream,
                     ttq_plan **out);
int ttq_batch_run(ttq_plan *batch, ttq_result *results /* [count] */);

/* Autotuner: times the evaluation, sample and rook kernels over `sweeps`
 * sweeps for candidate launch shapes (CTAs per instance of the rook kernels,
 * which spread all interfaces' work over one grid; CTAs per interface of the
 * sample kernel; CTAs per instance of the evaluation kernel; the largest rook
 * work item, 1, 2 or 4 rows of 32 candidates), keeps the fastest and writes
 * them to chosen[0..3] (rook, sample, eval, rook rows) if chosen != NULL.
 * Launch shapes never change results.  ttq_plan_set_config sets the CTA
 * counts directly (each in 1..65535) and ttq_plan_set_rook_rows the item size
 * (1, 2 or 4), else TTQ_ERR_INVALID_ARG. */
int ttq_batch_autotune(ttq_plan *plan, int sweeps, int32_t *chosen /* [4] */);

/* Concurrent groups of a batch run: the instances sorted by cost (rank cap^2
 * times the nodes of all modes, ties in instance order) are split into
 * `groups` contiguous groups of near-equal count, each a WHILE loop of its own
 * in the batch's run graph with no dependence on the others, so a group of
 * small instances does not wait for the sweeps of the large ones.  1..min(8,
 * count / 2); the default is min(8, count / 32) (at least 1).  Results are the
 * same for every grouping (each instance's kernels are the same). */
#define TTQ_MAX_BATCH_GROUPS 8
int ttq_batch_set_groups(ttq_plan *batch, int groups);
int ttq_plan_set_config(ttq_plan *plan, int rook_ctas, int sample_ctas, int eval_ctas);
int ttq_plan_set_rook_rows(ttq_plan *plan, int rows);

/* --- serving: continuous batching -----------------------------------------
 * A server owns a caller-allocated device pool (`pool`, pool_bytes, 256-byte
 * aligned; its size is the HBM admission budget) and at most max_slots
 * integrals in flight.  ttq_server_submit copies a request (host arrays) into
 * the server's arrival queue and returns its id; a request whose plan
 * footprint (ttq_workspace_bytes, reserved at its rank cap) exceeds the pool
 * is refused with TTQ_ERR_ADMISSION.  ttq_server_step, at a sweep boundary:
 * retires the requests that stopped (their memory returns to the pool, their
 * result becomes available) and admits queued requests in arrival order while
 * a slot and pool memory are free (how requests in flight run: see
 * ttq_server_set_mode).  Each
 * result equals what a single plan gives for the same problem, whatever else
 * is in flight.  ttq_server_poll returns TTQ_PENDING until a request is done;
 * ttq_server_drain returns up to max finished results at once.
 * ttq_server_stats: [in flight, queued, admitted, retired, sweeps run, free
 * pool bytes].  A server is not thread-safe. */
typedef struct ttq_server ttq_server;
int ttq_server_create(void *pool, size_t pool_bytes, int max_slots, void *stream, ttq_server **out);
int ttq_server_destroy(ttq_server *server);
int ttq_server_submit(ttq_server *server, const ttq_problem *p, uint64_t *request_id);
int ttq_server_step(ttq_server *server, int sweeps, int *in_flight, int *queued, int64_t *completed);
int ttq_server_poll(ttq_server *server, uint64_t request_id, ttq_result *out);
int ttq_server_drain(ttq_server *server, uint64_t *ids, ttq_result *results, int max, int *n);
int ttq_server_stats(const ttq_server *server, int64_t *stats /* [6] */);

/* Serving engine.  Mode 0 (the default): every request in flight is a plan of
 * its own over its pool region, its whole run one CUDA graph launch on one of
 * the server's 16 streams, so requests overlap on the device as they arrive;
 * ttq_server_step retires the requests whose runs have finished (waiting for
 * the earliest admitted one when none has) and admits queued ones; `sweeps`
 * is not used.  Mode 1: the requests in flight advance together, `sweeps`
 * sweeps per step, in the batched kernel launches (the batch form above).
 * Either way each result equals what a single plan gives for the problem.
 * Set before the first request is admitted. */
int ttq_server_set_mode(ttq_server *server, int mode);

/* --- stage-level entry points (replay and inspection) ------------------- */

/* Initial index set: the largest |A| among init_samples seeded random points. */
int ttq_plan_init(ttq_plan *plan);

/* Replace the index sets by the given nested sets in parent-pointer form
 * (Eq. 4): I<=k[a] = (I<=k-1[lpar[k-1][a]], lnode[k-1][a]) and
 * I>k[b] = (rnode[k-1][b], I>k+1[rpar[k-1][b]]), host arrays concatenated over
 * k = 1..d-1 with ranks[k] entries each (ranks has d+1 entries, ranks[0] =
 * ranks[d] = 1).  The next sweep re-evaluates every core and refactors every
 * cross matrix from scratch. */
int ttq_plan_set_state(ttq_plan *plan, const int32_t *ranks, const int32_t *lpar, const int32_t *lnode,
                       const int32_t *rpar, const int32_t *rnode);
int ttq_plan_get_state(ttq_plan *plan, int32_t *ranks, int32_t *lpar, int32_t *lnode,
                       int32_t *rpar, int32_t *rnode);

/* One sweep: evaluate the new core entries, factor the cross matrices,
 * contract the integral, then (search != 0) run Alg. 2 on every interface on
 * the sets of this sweep and append the accepted pivots (Alg. 6).  Writes the
 * sweep's integral to *value and, if pivots != NULL, d-1 ttq_pivot records.
 * In double-double mode with search == 0, *value / *value_lo are the
 * double-double contraction; with search != 0 the FP64 one.  No stopping rule
 * is applied.  With several pivots per sweep (npiv > 1) each record describes
 * the interface's first search and `accepted` is the number of pivots the
 * interface appended; the pivots themselves are the new rows of the nested
 * sets (ttq_plan_get_state). */
int ttq_plan_sweep(ttq_plan *plan, int sweep_index, int search, double *value, double *value_lo,
                   ttq_pivot *pivots);

/* Copy core k (1..d) Y_k = A(I<=k-1, i_k, I>k) to host memory as a dense
 * row-major r_{k-1} x N_k x r_k array (valid after a sweep). */
int ttq_plan_get_core(ttq_plan *plan, int k, double *host_out);

/* Weighted tensor entries A = prod_k w_k[i_k] g(t) (no family constant) at
 * npts multi-indices idx (device, row-major npts x d int32) into out (device
 * npts doubles), on the plan's stream. */
int ttq_plan_eval_points(ttq_plan *plan, const int32_t *idx, int64_t npts, double *out);

/* Number of the library's kernel launches issued by this plan so far. */
int64_t ttq_plan_launches(const ttq_plan *plan);

/* Graph execution on (default, except on the legacy default stream) or off:
 * off, every kernel of a sweep is a plain stream launch and the host checks
 * the stopping flag every two sweeps (same work and results; for profilers
 * that replay individual launches). */
int ttq_plan_set_graphs(ttq_plan *plan, int enable);

/* Search of a sweep (Alg. 2 on every interface, Alg. 6): mode 0 (the
 * default) as separate launches per stage (samples, 3 x (column step,
 * decisions, row step, decisions)), the form batches always use; mode 1
 * (single-instance plans only) as one persistent kernel in which every
 * interface owns a group of CTAs and hands its stages on through flags in
 * device memory, without kernel boundaries.  Both compute the same values bit
 * for bit.  ttq_plan_set_wait_limit bounds every
 * wait between CTAs of the persistent search (nanoseconds of the GPU's global
 * timer, default 1 s); a wait that passes it ends the run with
 * TTQ_ERR_TIMEOUT and leaves the plan usable. */
int ttq_plan_set_search(ttq_plan *plan, int mode);

/* Sweep kind: 0 (default) the dimension-parallel sweep of Alg. 6, every
 * interface searched on the index sets of the previous sweep and all pivots
 * appended at the end; 1 the sequential left-to-right sweep of Alg. 5, the
 * paper's single-process comparison: interface k's superblock is built from
 * I<=k-1 as interface k-1's step just extended it, and each pivot is appended
 * at once.  Single-instance plans only; runs with plain launches (no CUDA
 * graph).  ttq_plan_sweep then reports no per-interface pivots. */
int ttq_plan_set_sequential(ttq_plan *plan, int enable);
int ttq_plan_set_wait_limit(ttq_plan *plan, uint64_t ns);

/* Bytes this plan has copied host->device (problem inputs, descriptor) and
 * device->host (state and flags read back) since it was created. */
int ttq_plan_transfer_bytes(const ttq_plan *plan, int64_t *h2d, int64_t *d2h);

/* Per-kernel timing.  With timing enabled every launch of a sweep is
 * bracketed by CUDA events on the plan's stream; ttq_plan_kernel_times writes,
 * for each of the TTQ_NUM_KERNELS kernel kinds (index order: eval_slabs, qr
 * (both halves of the QR update), contract, samples, rook_col, rook_row,
 * update (the search's last decisions launch, which also ends the sweep),
 * init, setup, solve (the other decisions launches), search (the persistent
 * search, whose FP64 operations count under samples, rook_col, rook_row and
 * solve)), the summed
 * device time in ms and the launch count since the last reset, and the
 * algorithmic FP64 operations the kernel has done since the plan's state was
 * last set (cumulative; a division, exp or cosh counts as one operation, an
 * FMA as two).  Any output array may be NULL.  Synchronizes the stream. */
#define TTQ_NUM_KERNELS 11
int ttq_plan_set_timing(ttq_plan *plan, int enable);
int ttq_plan_kernel_times(ttq_plan *plan, double *ms, int64_t *launches, double *flops, int reset);

/* Whole integral without allocating anything, for callers that must not call
 * cudaMalloc (code running under another component's memory pool or a fixed
 * memory budget, plugins handed only a stream, paths that must not fail on
 * allocation).  The paper has no counterpart: this is a deployment variant of
 * ttq_plan_create + ttq_plan_run.
 *  - Device scratch: one fixed array of TTQ_NOALLOC_SCRATCH_BYTES (16 MiB),
 *    declared in the library, which every GPU that loads the library holds
 *    until the process exits.  A problem whose plan needs more
 *    (ttq_workspace_bytes) is rejected with TTQ_ERR_WORKSPACE.
 *  - nodes/weights must be host arrays (inputs_on_device == 0).
 *  - Every call looks up the scratch's device address (cudaGetSymbolAddress,
 *    which allocates nothing) with the caller's device current, so calls
 *    after a device reset or on another device find their own scratch; make
 *    the first call of the process before any stream capture starts (the
 *    first lookup may load the library's device code).
 *  - The call waits for its stream and copies from host memory on its own
 *    stack; on a stream that is capturing it returns TTQ_ERR_INVALID_ARG
 *    before doing any CUDA work, so the caller's capture is left intact.
 *  - Every call on a device uses the same scratch, which keeps the previous
 *    call's contents (the call resets what it reads).  Calls that overlap on
 *    the GPU (other streams, other host threads) race on it: serialize them.
 *  - Blocks until the result is on the host.  Same result as
 *    ttq_plan_create + ttq_plan_run on the same problem and stream. */
#define TTQ_NOALLOC_SCRATCH_BYTES (16u << 20)
int ttq_integrate_noalloc(const ttq_problem *p, void *stream, ttq_result *out);

const char *ttq_status_string(int status);
const char *ttq_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TTQ_H */
