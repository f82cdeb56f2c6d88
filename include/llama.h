/*
 * llama.h -- C ABI of the B300-native scheduling step of Llama
 * (arXiv 2102.01887): per-invocation slack (Section 4.1, Algorithm 1) and
 * cost-based configuration selection (Section 4.2, Eq. 1).
 *
 * Units and types.  Latencies are int32 microseconds, costs int64
 * nano-dollars per invocation (the C(x)/B(x) term of Eq. 1), times int64
 * microseconds.  All integer arithmetic is exact: decisions are bit-exact
 * against a plain CPU evaluation of the same definitions.
 *
 * Ownership.  Every llama_set_* call copies its (host) arrays into
 * library-owned device memory; the caller may free them on return.  The
 * scheduling calls read caller buffers and write the caller-owned output;
 * nothing the caller passes is retained after the call (blocking form) or
 * after the stream reaches the call (asynchronous form).
 *
 * Errors.  Every call returns an int status (LLAMA_OK or a negative
 * LLAMA_E* code); llama_last_error() gives a one-line description of the
 * last failure on that context.  A context is not thread-safe: use one
 * context per host thread, or serialise calls.
 */
#ifndef LLAMA_H
#define LLAMA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LLAMA_OK 0
#define LLAMA_EINVAL (-1)    /* invalid argument, table, DAG or invocation */
#define LLAMA_ENOMEM (-2)    /* device or host allocation failed */
#define LLAMA_ECUDA (-3)     /* a CUDA runtime call or kernel launch failed */
#define LLAMA_ENOTREADY (-4) /* scheduling before both DAGs and profiles are set */
#define LLAMA_ETIMEOUT (-5)  /* a bounded device-side wait gave up */

/* Objective (Section 4.2).  COST_FIRST: feasible (L < slack) beats
 * infeasible; among feasible configurations the lowest C/B wins, among
 * infeasible ones the lowest latency; ties go to the lowest configuration
 * index.  ALPHA: Eq. 1 in integers, obj = C/B if L < slack, otherwise
 * C/B + floor(alpha_num*L*R(x) / (alpha_den*B(x)*R_total(lambda(x)))),
 * saturating at INT64_MAX; argmin over (obj, index). */
#define LLAMA_MODE_COST_FIRST 0
#define LLAMA_MODE_ALPHA 1

/* llama_decision.flags */
#define LLAMA_FLAG_FEASIBLE 1 /* the chosen configuration meets its slack */
#define LLAMA_FLAG_INVALID 2  /* the invocation was rejected; cfg = -1 */
#define LLAMA_FLAG_TIMEOUT 4  /* not decided: a bounded device wait of the call gave up
                                 (the call reports LLAMA_ETIMEOUT); cfg = -1 */

/* Limits enforced by validation. */
#define LLAMA_MAX_HW 8          /* backends lambda */
#define LLAMA_MAX_CFG 8192      /* configurations of one operation */
#define LLAMA_MAX_INV (1 << 30) /* invocations in one call */
#define LLAMA_MAX_ALPHA 65535   /* alpha_num, alpha_den, B(x), R(x) upper bound */

typedef struct llama_ctx llama_ctx;

typedef struct llama_opts {
    int32_t mode;      /* LLAMA_MODE_* */
    int32_t n_hw;      /* number of backends, 1..LLAMA_MAX_HW */
    int64_t alpha_num; /* alpha = alpha_num / alpha_den, each in 1..LLAMA_MAX_ALPHA (ALPHA mode) */
    int64_t alpha_den;
    int32_t device;    /* CUDA device ordinal the context lives on */
    int32_t use_graph; /* nonzero: replay each scheduling call as one CUDA graph */
} llama_opts;

/* One scheduling decision; 24 bytes, naturally aligned. */
typedef struct llama_decision {
    int32_t cfg;   /* op-local index of the chosen configuration, -1 if invalid */
    int32_t lat;   /* L(cfg), us */
    int64_t cost;  /* C(cfg)/B(cfg), nano-dollars */
    int32_t slack; /* slack(op, lambda(cfg)), us (Algorithm 1) */
    int32_t flags; /* LLAMA_FLAG_* */
} llama_decision;

/* Create a context on opts->device: the state of one Configurator (Section
 * 4: the Logic Plane's slack allotment, Algorithm 1, and cost-based
 * optimizer, Eq. 1), with the objective of Eq. 1 chosen by opts->mode and
 * alpha = alpha_num / alpha_den.  *out is set on success (the caller owns
 * the context and releases it with llama_destroy).
 * Errors: EINVAL (bad opts), ENOMEM, ECUDA. */
int llama_create(llama_ctx **out, const llama_opts *opts);

/* Release every device and host resource of the context (NULL is a no-op). */
void llama_destroy(llama_ctx *ctx);

/* Pipelines (Section 3.2, Fig. 1): n_dags DAGs over global operation ids.
 *   dag_op_off[n_dags+1]  DAG d owns global ops [dag_op_off[d], dag_op_off[d+1]);
 *                         dag_op_off[0] = 0, every DAG has at least one op.
 *   row_ptr[n_ops+1]      successor CSR, n_ops = dag_op_off[n_dags];
 *   col[row_ptr[n_ops]]   successor global ids, inside the op's own DAG;
 *   slo_us[n_dags]        pipeline latency target, 1..INT32_MAX.
 * Host memory.  Rejects (EINVAL) a malformed CSR, a cross-DAG edge, a
 * self-loop or a cycle.  Replaces any previous DAGs. */
int llama_set_dags(llama_ctx *ctx, int32_t n_dags, const int32_t *dag_op_off,
                   const int32_t *row_ptr, const int32_t *col, const int64_t *slo_us);

/* Profiles (Section 3.2, "configuration specification"; Section 4.2).
 *   cfg_off[n_ops+1]          configurations of op v are [cfg_off[v], cfg_off[v+1]),
 *                             1..LLAMA_MAX_CFG per op;
 *   hw_off[n_ops*(n_hw+1)]    op-local start of each backend's segment: configurations
 *                             are grouped hardware-major, hw_off[v][0] = 0,
 *                             non-decreasing, hw_off[v][n_hw] = size of op v;
 *   lat_us[n_cfg]             L(x), 1..INT32_MAX-1;
 *   cost_nd[n_cfg]            C(x)/B(x), >= 0;
 *   ref_cfg[n_ops]            op-local reference configuration (Section 3.2:
 *                             smallest CPU configuration, 1 core, batch 1);
 *   batch, res [n_cfg]        B(x), R(x) in 1..LLAMA_MAX_ALPHA   (ALPHA mode; else NULL ok);
 *   res_total[n_hw]           R_total(lambda) in 1..INT32_MAX     (ALPHA mode; else NULL ok).
 * Host memory.  Copies the tables to the device and builds the scan
 * encoding there.  Errors: EINVAL, ENOMEM, ECUDA. */
int llama_set_profiles(llama_ctx *ctx, int32_t n_ops, const int64_t *cfg_off,
                       const int32_t *hw_off, const int32_t *lat_us, const int64_t *cost_nd,
                       const int32_t *ref_cfg, const int32_t *batch, const int32_t *res,
                       const int32_t *res_total);

/* Queueing time per backend, queueingTime(lambda) of Algorithm 1 (Eq. 2's
 * value, supplied by the caller), q_us[n_hw] in 0..INT32_MAX; host memory;
 * default all zero. */
int llama_set_queue(llama_ctx *ctx, const int64_t *q_us);

/* Feedback (Section 3.3: the Manager records every executed invocation's
 * latency and cost and updates the profiles by exponential smoothing): n
 * observations (global operation op[i], op-local configuration cfg[i],
 * measured lat_us[i] >= 1 and cost_nd[i] >= 0) update the tables in place,
 *   L <- ((beta_den - beta_num) L + beta_num L_obs + beta_den / 2) / beta_den
 * in exact integers (the same for the cost), a configuration's observations
 * applied in their order; 0 <= beta_num <= beta_den <= 65535.  The encodings
 * of the touched operations are rebuilt on the device, on `stream`; calls
 * enqueued after it on that stream, and the blocking calls of this context,
 * see the new tables (the critical paths follow the new reference latencies);
 * calls on other streams must be ordered after it by the caller.  Invalid observations are skipped and counted into
 * *rejected (device int64, nullable).  Device pointers.  Errors: EINVAL,
 * ENOTREADY, ENOMEM, ECUDA. */
int llama_feedback(llama_ctx *ctx, int64_t n, const int32_t *op, const int32_t *cfg, const int32_t *lat_us,
                   const int64_t *cost_nd, int32_t beta_num, int32_t beta_den, int64_t *rejected,
                   void *stream);

/* Eq. 3, per-backend minima (Section 4.4): for every invocation i and backend
 * h, the least Eq. 1 objective (the numeric one, with the context's alpha:
 * C/B if L < slack(op, h), else C/B + floor(alpha_num L R / (alpha_den B
 * R_total(h))), saturating) among op's configurations on h -- INT64_MAX for an
 * empty backend or an invalid invocation -- into obj_min[i * n_hw + h]
 * (device int64).  Arguments as llama_schedule_async.  Needs batch, res and
 * res_total in the profiles.  Errors: EINVAL, ENOTREADY, ECUDA. */
int llama_backend_objectives(llama_ctx *ctx, int64_t n_inv, const int32_t *dag, const int32_t *op_local,
                             const int64_t *start_us, int64_t now_us, int64_t *obj_min, void *stream);

/* Priority-based commit (Section 4.4): the order to commit n decided
 * invocations (dag, op_local, dec as scheduled; obj_min from
 * llama_backend_objectives) into the backends' commit queues: by the backend
 * of each decision, then by descending affinity of the invocation's operation
 * to that backend (Eq. 3: the least objective on the other backends over the
 * least on its own; +inf when its own is 0), then by index; invalid decisions
 * last.  order (device int32 [n]) receives invocation indices; affinity
 * (device double [n], nullable) each invocation's affinity.  Errors: EINVAL,
 * ENOTREADY, ENOMEM, ECUDA. */
int llama_commit_order(llama_ctx *ctx, int64_t n, const int32_t *dag, const int32_t *op_local,
                       const llama_decision *dec, const int64_t *obj_min, int32_t *order, double *affinity,
                       void *stream);

/* The current latency and cost tables (host arrays of n_cfg; blocking). */
int llama_get_profiles(llama_ctx *ctx, int32_t *lat_us, int64_t *cost_nd);

/* Queueing time of every backend from the invocations queued on it (Eq. 2,
 * Section 4.3): Q[lambda] = floor(sum over queued i with lambda(x_i) = lambda
 * of L(x_i) R(x_i) / R_total(lambda)) -- the exact integer sum, floored once --
 * from the n decided invocations (dag[i], op_local[i], dec[i]: decisions of
 * earlier scheduling calls, e.g. the speculative and commit queues; invalid
 * ones are skipped) and the profiles' resources.  Written to q_out (device,
 * n_hw int64, nullable); with apply != 0 it also becomes the context's
 * queueing time for later calls, on the device (no host round trip): calls
 * after it on `stream`, and the blocking calls of this context; calls on
 * other streams must be ordered after it by the caller.  Device
 * pointers, enqueued on `stream`.  Errors: EINVAL (arguments, or profiles set
 * without res / res_total), ENOTREADY. */
int llama_queue_time(llama_ctx *ctx, int64_t n, const int32_t *dag, const int32_t *op_local,
                     const llama_decision *dec, int64_t *q_out, int32_t apply, void *stream);

/* Schedule n_inv pending invocations at time now_us (blocking): for each,
 * its slack on every backend (Section 4.1, Algorithm 1: the target minus the
 * elapsed time and the backend's queueing time, times the op's share of its
 * longest remaining reference path) and the configuration that Eq. 1
 * (Section 4.2) selects against the slack of the configuration's own backend.
 *   dag[n_inv], op_local[n_inv]  the invocation's DAG and op-local operation;
 *   start_us[n_inv]              start time of its pipeline instance, 0..now_us;
 *   out[n_inv]                   decisions, written in invocation order.
 * Each pointer may be host or device memory (detected per pointer); inputs
 * in page-locked host memory are read in place by the kernels, pageable ones
 * are copied to the device first.  The arrays must not change during the
 * call.  An invalid invocation (bad DAG or op index, start outside 0..now) gets
 * cfg = -1 and LLAMA_FLAG_INVALID, every valid one is still decided, and the
 * call returns EINVAL.  n_inv = 0 is a no-op.  Errors: EINVAL, ENOTREADY,
 * ENOMEM, ECUDA. */
int llama_schedule(llama_ctx *ctx, int64_t n_inv, const int32_t *dag, const int32_t *op_local,
                   const int64_t *start_us, int64_t now_us, llama_decision *out);

/* Same as llama_schedule (Algorithm 1 and Eq. 1, Sections 4.1-4.2),
 * enqueued on `stream` (a cudaStream_t; NULL = the legacy default stream)
 * and returning without waiting.  Every pointer must
 * be device memory that stays valid until the stream passes the call.
 * Invalid invocations are flagged in `out` but the return value does not
 * report them.  Scratch space is library-owned and grows on demand; call
 * llama_reserve first to keep allocations out of the call (for instance
 * before a stream capture).  The calls of one context share that scratch:
 * enqueue them on one stream, or order them, so that no two run at once.
 * Each call leaves the scratch's counters cleared for the next one, so a
 * call enqueues kernels only (no memset).  Errors: EINVAL (bad arguments),
 * ENOTREADY, ENOMEM, ECUDA. */
int llama_schedule_async(llama_ctx *ctx, int64_t n_inv, const int32_t *dag,
                         const int32_t *op_local, const int64_t *start_us, int64_t now_us,
                         llama_decision *out, void *stream);

/* Workspaces: the scratch of one scheduling call, separate from the
 * context's own, so that calls of one context run concurrently on several
 * streams (each call with its own workspace, no two calls on one workspace at
 * once) while sharing the context's read-only tables.  A workspace holds
 * calls of up to max_inv invocations for the context's current profiles; new
 * profiles with more operations need a new workspace.  Errors: EINVAL,
 * ENOTREADY, ENOMEM, ECUDA. */
typedef struct llama_ws llama_ws;
int llama_ws_create(llama_ctx *ctx, int64_t max_inv, llama_ws **out);
void llama_ws_destroy(llama_ws *ws);

/* llama_schedule_async with the workspace ws (direct launches, no graph).
 * Each pointer may be device memory or page-locked host memory: host inputs
 * are read in place by the kernels over the host link; for a host `out` the
 * decisions go to a device buffer of the workspace (allocated by the first
 * such call, max_inv records) and are copied back on `stream`.  So a caller
 * holding host arrays can keep several calls in flight on several streams
 * (one workspace each), one call's copy back overlapping the next one's reads.
 * Pageable host memory is refused (EINVAL).  Host arrays must stay valid and
 * unchanged until the stream passes the call. */
int llama_schedule_ws_async(llama_ctx *ctx, llama_ws *ws, int64_t n_inv, const int32_t *dag,
                            const int32_t *op_local, const int64_t *start_us, int64_t now_us,
                            llama_decision *out, void *stream);

/* How the workspace's calls take inputs in page-locked host memory: read in
 * place by the kernels over the host link (LLAMA_WS_INPUTS_IN_PLACE, the
 * default; the fastest for a call alone) or copied into the workspace by the
 * copy engine on the call's stream first (LLAMA_WS_INPUTS_COPY: the kernels
 * then do not wait on the link, so with calls in flight on several streams
 * one call's inputs, another's kernels and a third's decisions can move at
 * once).  The copy buffers (16 B per invocation of max_inv) are allocated by
 * the first call that needs them.  Errors: EINVAL. */
#define LLAMA_WS_INPUTS_IN_PLACE 0
#define LLAMA_WS_INPUTS_COPY 1
int llama_ws_set_inputs(llama_ws *ws, int32_t mode);

/* Status of the workspace's last completed call (read once the stream has
 * passed it; blocking): the number of invalid invocations, and whether a
 * bounded device wait gave up. */
int llama_ws_status(llama_ws *ws, int64_t *invalid, int32_t *timeout);

/* Allocation-free variant of llama_schedule_async.  The paper has no
 * counterpart: this is a deployment convenience.  Some callers cannot let a
 * library call cudaMalloc or cudaFree while they schedule: a serving loop
 * whose device memory is carved up front by its own allocator, a
 * latency-bound loop that cannot take the implicit synchronisation of the
 * CUDA allocator, or code running where the allocator must not be entered.
 * This call allocates nothing: its bucketing scratch is one fixed, file-scope
 * device array of about 4.2 MB, which every GPU that loads the library holds
 * until the process exits.  Same arguments and results as
 * llama_schedule_async (device pointers, enqueued on `stream`, invalid
 * invocations flagged in `out`), with these limits: n_inv at most
 * LLAMA_STATIC_MAX_INV and at most LLAMA_STATIC_MAX_OPS operations in the
 * profiles; larger sizes are rejected with EINVAL before anything is
 * launched.  The first call on a device looks up the array's device address
 * (once per device, with that device current); make that first call before
 * any stream capture.  The address stays cached for the process: after
 * cudaDeviceReset (or anything else that destroys the device's primary
 * context) this entry point must not be called again in that process.
 * Every call shares the one array, which keeps the last call's contents.
 * The counters and control words a call needs at zero are zero when it
 * starts: the array starts zeroed, every completed call leaves them cleared
 * (its last kernel clears them), and a call whose later launch fails clears
 * them with memsets on its stream before returning ECUDA.  Calls that overlap
 * on the GPU race on the array: serialise them.  A bounded device wait that
 * gives up, and invalid invocations, are not reported by the return value
 * (the call returns once its kernels are enqueued): read them with
 * llama_static_status.  llama_last_launch_count reports this call's kernels.
 * Errors: EINVAL, ENOTREADY, ECUDA. */
#define LLAMA_STATIC_MAX_INV 65536
#define LLAMA_STATIC_MAX_OPS 4096
int llama_schedule_static(llama_ctx *ctx, int64_t n_inv, const int32_t *dag,
                          const int32_t *op_local, const int64_t *start_us, int64_t now_us,
                          llama_decision *out, void *stream);

/* Status of the last llama_schedule_static call completed on the context's
 * device (no counterpart in the paper): the number of invalid invocations
 * and whether a bounded device wait gave up (then every valid invocation of
 * that call is flagged LLAMA_FLAG_TIMEOUT with cfg = -1).  Enqueues a copy of
 * the array's two status words on `stream` (order it after the call) and
 * waits for it; allocates nothing.  invalid and timeout are host pointers,
 * each nullable.  Errors: EINVAL (a null context, a device ordinal above 63),
 * ENOTREADY, ECUDA. */
int llama_static_status(llama_ctx *ctx, void *stream, int64_t *invalid, int32_t *timeout);

/* Launch schedule of the scoring kernel (no counterpart in the paper; a
 * B300 schedule that changes speed, never results):
 *   lanes_min_vectors  each of the lanes sharing one invocation scans at least
 *                      this many 8-configuration vectors, 1..1024 (default 16);
 *   inv_per_thread     invocations a thread scores together against each staged
 *                      vector: 1, 2 or 4 (default 2);
 *   chunk_entries      table entries staged in shared memory at a time: a
 *                      multiple of 8 in 8..LLAMA_MAX_CFG + 8*LLAMA_MAX_HW (the
 *                      largest padded table), or 0 for the default (the largest
 *                      padded table in the fewest even pieces of about 4096);
 *   stages             staging buffers per CTA: 1 (tiles claimed from a
 *                      counter as CTAs finish; default) or 2 (tiles taken
 *                      round-robin, the next chunk copied while one is scored).
 * Call after llama_set_profiles (which resets the chunk to its default).
 * Errors: EINVAL, ENOTREADY (no profiles), ECUDA. */
int llama_set_tuning(llama_ctx *ctx, int32_t lanes_min_vectors, int32_t inv_per_thread,
                     int32_t chunk_entries, int32_t stages);

/* Distinct latencies of an operation staged in shared memory by the scoring
 * kernel (no counterpart in the paper; changes speed, never results): an op
 * with at most max_entries of them (1..LLAMA_MAX_CFG; default 4096) has its
 * sorted list copied beside its table and searched there; an op with more is
 * counted by the count pass or searched in global memory.  Staging a list
 * costs 4 B per distinct latency per tile: worth it where an op's table serves
 * many invocations, not where tables stream from DRAM for a few each.  Call
 * after llama_set_profiles (which resets it to 4096).  Errors: EINVAL,
 * ENOTREADY (no profiles), ECUDA. */
int llama_set_dlat_stage(llama_ctx *ctx, int32_t max_entries);

/* Persistent CTAs of the scoring kernel per SM (no counterpart in the paper;
 * changes speed, never results): 0 (default) as many as its registers and
 * shared memory allow, else at most ctas_per_sm (1..32).  Fewer, larger
 * shares of the SM can be faster where staging and scanning contend; more
 * CTAs keep more table copies in flight where tables stream from DRAM.
 * Call after llama_set_profiles (which resets it to 0).  Errors: EINVAL,
 * ENOTREADY (no profiles), ECUDA. */
int llama_set_score_occupancy(llama_ctx *ctx, int32_t ctas_per_sm);

/* Count pass of the scan method (no counterpart in the paper; changes speed,
 * never results).  Operations with more distinct latencies than the scoring
 * kernel stages in shared memory need, per invocation and backend, the number
 * of them below the slack (the feasibility threshold of Eq. 1 in latency-rank
 * form).  ON: a separate kernel between bucketing and scoring computes these
 * counts, one thread per invocation (a probe line, a second-level probe line
 * and a short bisection per backend); OFF: the scoring kernel searches them
 * itself, a warp-wide search per (invocation, backend), overlapped with the
 * staging of the table.  AUTO (default): ON when at least half of the
 * operations have padded tables larger than the staged distinct latencies.
 * The pass is launched only while some operation can have more distinct
 * latencies than are staged (they are at most its configurations, which
 * feedback can reach), never by llama_schedule_static.  Errors: EINVAL. */
#define LLAMA_COUNT_PASS_AUTO 0
#define LLAMA_COUNT_PASS_ON 1
#define LLAMA_COUNT_PASS_OFF 2
int llama_set_count_pass(llama_ctx *ctx, int32_t mode);

/* Method of the selection step (a4).  SCAN (default): every configuration of
 * the invocation's operation is scored (Eq. 1, Section 4.2), tables staged
 * through shared memory and shared by the op's invocations.  STAIRCASE: an
 * exact rearrangement of the same argmin that the paper does not describe:
 * per operation and backend, the configurations sorted by latency, and at
 * every latency rank k the best key among those below k (the feasible branch)
 * and, in ALPHA mode, among those at or above k (the infeasible branch), built
 * once from the profiles (16-bit keys, n_hw * (distinct latencies + 1) per
 * operation).  A decision is then one search per backend and n_hw lookups
 * instead of a scan.  Decisions are identical under both methods.  Setting
 * STAIRCASE builds its tables (again after every llama_set_profiles).
 * Errors: EINVAL, ENOMEM, ECUDA. */
#define LLAMA_METHOD_SCAN 0
#define LLAMA_METHOD_STAIRCASE 1
int llama_set_method(llama_ctx *ctx, int32_t method);

/* Small calls of the SCAN method (no counterpart in the paper; changes speed,
 * never results): a call of at most n_inv invocations (default
 * LLAMA_DIRECT_DEFAULT) skips the bucketing by operation.  Two kernels instead
 * of the bucketing and scoring kernels: the critical paths of every DAG
 * (Algorithm 1's longest remaining path), then a warp per invocation that
 * computes its slack per backend and scans its operation's rank-encoded table
 * straight from L2 (Eq. 1), with the same decisions.  Such a call has no
 * bounded wait, so it never times out.  With few invocations per operation no
 * table copy is shared, and two short kernels replace a cooperative launch and
 * its grid barrier.  0: every call is bucketed.  Errors: EINVAL (n_inv outside
 * 0..LLAMA_DIRECT_LIMIT). */
#define LLAMA_DIRECT_DEFAULT 1024
#define LLAMA_DIRECT_LIMIT (1 << 20)
int llama_set_direct_max(llama_ctx *ctx, int64_t n_inv);

/* Bounded device waits (no counterpart in the paper).  The bucketing kernel's
 * grid barriers poll at most `tries` times before they give up: the call then
 * decides nothing (every valid invocation is flagged LLAMA_FLAG_TIMEOUT with
 * cfg = -1) and reports LLAMA_ETIMEOUT (llama_schedule), or through
 * llama_ws_status / llama_static_status.  The default,
 * LLAMA_WAIT_LIMIT_DEFAULT, is never reached by a launch whose blocks are all
 * resident; a lower value (0: give up at once) exercises the give-up path.
 * Table staging waits keep their own fixed bound.  Calls small enough for
 * the path without bucketing (llama_set_direct_max) have no wait to give up.
 * Errors: EINVAL (tries outside 0..LLAMA_WAIT_LIMIT_DEFAULT). */
#define LLAMA_WAIT_LIMIT_DEFAULT (1 << 20)
int llama_set_wait_limit(llama_ctx *ctx, int32_t tries);

/* Pre-allocate scratch for calls of up to max_inv invocations. */
int llama_reserve(llama_ctx *ctx, int64_t max_inv);

/* Longest remaining reference-latency path of every operation, op included
 * (the RemainingPathLatency maximised over the paths of Algorithm 1):
 * cp_us[n_ops], host memory.  Runs the device critical-path pass. */
int llama_critical_path(llama_ctx *ctx, int64_t *cp_us);

/* Slack of every invocation for every backend (Algorithm 1; 0 once the
 * target has passed), slack_us[n_inv*n_hw] int32, row-major by invocation,
 * -1 for an invalid invocation.  Host or device pointers, blocking. */
int llama_slack(llama_ctx *ctx, int64_t n_inv, const int32_t *dag, const int32_t *op_local,
                const int64_t *start_us, int64_t now_us, int32_t *slack_us);

/* Tracing.  events[0..LLAMA_TRACE_EVENTS-1] are caller-owned cudaEvent_t
 * handles; once set, every scheduling call records them on its stream at
 * the phase boundaries: [0] call start, [1] after the bucketing kernel
 * (critical path, counting per operation, bucket layout, slack), [2] after
 * the scoring kernel (and the count pass before it, when it runs).  Traced calls launch their kernels directly (no CUDA
 * graph) and the scoring kernel no longer overlaps the end of the bucketing
 * kernel.  n_events = 0 turns tracing off.  The events must stay valid while
 * tracing is on.  Errors: EINVAL. */
#define LLAMA_TRACE_EVENTS 3
int llama_set_trace_events(llama_ctx *ctx, void *const *events, int32_t n_events);

/* Per-call statistics (no counterpart in the paper): once set, every blocking
 * llama_schedule call appends one JSON object per line to the file at path
 * (opened for appending; NULL or "" closes it): the call's index, n_inv,
 * now_us, method, kernel launches, whether a CUDA graph was replayed, the
 * invalid count, whether a bounded wait gave up, the device time of its
 * kernels (events around them), the host time of the whole call, invocations
 * per second of device time, and -- when the decisions are written to host
 * memory -- how many were feasible (met their target) and, with the
 * invocations in host memory too, how many configurations the decided ones
 * scored and per second of device time (null otherwise).  Errors: EINVAL (the
 * file cannot be opened), ECUDA. */
int llama_set_stats_file(llama_ctx *ctx, const char *path);

/* Checked build (no counterpart in the paper).  A library compiled with
 * -DLLAMA_CHECK bounds-checks the indices its kernels compute (bucket
 * positions, tile entries, staged table ranges, count-pass positions, decode
 * keys, serving-loop slots); a failed check sets its bit in the context's
 * check word and skips the access (never a trap), so the call completes with
 * a wrong result that the word reports.  llama_check_build returns 1 in such
 * a build and 0 otherwise; llama_check_word copies the word into *bits
 * (blocking; all zero in a normal build) and clears it when clear != 0.
 * Errors: EINVAL, ECUDA. */
#define LLAMA_CHECK_SCATTER 1u
#define LLAMA_CHECK_TILE 2u
#define LLAMA_CHECK_STAGE 4u
#define LLAMA_CHECK_COUNTS 8u
#define LLAMA_CHECK_DECODE 16u
#define LLAMA_CHECK_LOOP 32u
int llama_check_build(void);
int llama_check_word(llama_ctx *ctx, uint32_t *bits, int32_t clear);

/* Kernel launches issued by the last scheduling call (for accounting). */
int llama_last_launch_count(llama_ctx *ctx);

/* Stragglers and failures (Section 3.4, "Handling stragglers and invocation
 * failures"; time-out of Section 5): which of n invocations, decided at now_us
 * with decisions dec[i], get a duplicate invocation, and when the duplicate is
 * handed back to slack allotment and configuration.  Invocation i ran for
 * obs_us[i] >= 0 microseconds after now_us and then completed, or then
 * reported an error (failed[i] != 0; failed may be NULL: no errors).  Its
 * time-out is ceil(timeout_num * dec[i].lat / timeout_den) us (3/2 in the
 * paper).  A duplicate is made when the error arrives no later than the
 * time-out, or when the invocation is still running at the time-out; it is
 * handed back at the first multiple of tick_us (the Manager's check period) at
 * or after now_us + that moment.  Undecided invocations (cfg < 0) get none.
 * Writes the duplicates' indices to dup_idx and their hand-back times to
 * resubmit_us (each at most n long, host), their number to *n_dup.  Rescheduled
 * with the invocation's own start time at the later now, a duplicate gets no
 * more slack on any backend than the original (Algorithm 1: less of the target
 * is left).  Host memory and host code only.  Errors: EINVAL. */
int llama_stragglers(int64_t n, const llama_decision *dec, const int64_t *obs_us, const uint8_t *failed,
                     int64_t now_us, int32_t timeout_num, int32_t timeout_den, int64_t tick_us,
                     int64_t *dup_idx, int64_t *resubmit_us, int64_t *n_dup);

/* Measured ceiling of the scan's inner loop (no counterpart in the paper; the
 * denominator of the scoring kernel's ALU roofline): the rate at which the
 * device issues the scan's instruction mix for two configurations -- one
 * packed subtract of latency ranks, one LOP3, one per-half 16-bit minimum
 * (LLAMA_MODE_COST_FIRST), plus one PRMT (LLAMA_MODE_ALPHA) -- on operands
 * already in registers, on every SM.  *scores_per_s receives configurations
 * per second: the best of 20 timed launches after 40 untimed ones (about
 * 25 ms of full load, so the SM clock has left any idle state).  Allocates a
 * 16-byte buffer for the duration of the call.  Errors: EINVAL, ECUDA. */
int llama_alu_peak(int32_t device, int32_t mode, double *scores_per_s);

/* Measured floor of the bucketing step's per-op counting (no counterpart in the
 * paper; reported beside the bucketing kernel's roofline): n operation indices
 * spread by a hash over n_counters counters one 128-byte line apart, loaded
 * coalesced, counted with returning atomic adds, four in flight per thread, on
 * as many blocks as the bucketing kernel runs (four per SM), every rank stored
 * -- the counting pattern of the bucketing kernel, alone.  *atomic_us receives
 * the best time of that kernel, *stream_us the best time of the same loads and
 * stores without the atomics (10 timed launches each, after warm-up ones).
 * Allocates 8 * n + 128 * n_counters bytes for the duration of the call.
 * n in 1..LLAMA_MAX_INV, n_counters >= 1.  Errors: EINVAL, ECUDA. */
int llama_count_rate(int32_t device, int64_t n, int32_t n_counters, double *atomic_us, double *stream_us);

/* One-line description of the last error on ctx (never NULL). */
const char *llama_last_error(llama_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LLAMA_H */
