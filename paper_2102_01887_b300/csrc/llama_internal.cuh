// llama_internal.cuh -- device-side data layout and kernel entry points of
// the scheduling step (Section 4.1 Algorithm 1, Section 4.2 Eq. 1).
//
// Layout in HBM (all library-owned, written by llama_set_*):
//   DAGs      dag_op_off[n_dags+1], row_ptr[n_ops+1], col[n_edges], slo[n_dags],
//             topo[n_ops] (ops of each DAG ordered by height above the sinks),
//             lvl_off[n_levels+1] (ranges of topo per height), dag_lvl[n_dags+1].
//   Profiles  cfg_off[n_ops+1] int64, hw_off[n_ops*(H+1)], lat[n_cfg] int32,
//             cost[n_cfg] int64, ref_cfg[n_ops] (+ batch, res, res_total).
//   Scan encoding (built on the device by the encode kernels):
//             pad_off[n_ops+1] int64   start of op v in the padded space, a multiple of 8;
//             seg_pad[n_ops*(H+1)]     op-local padded start of each backend segment,
//                                      every segment padded to a multiple of 8 entries;
//             dlat[n_pad] int32        the op's distinct latencies, ascending, at
//                                      pad_off[v] (dlat_n[v] of them);
//             lrb[n_pad] u16           0x8000 + rank of L(x) among the op's distinct
//                                      latencies (kLatRankPad at pads), so that
//                                      L(x) < s  <=>  rank < #(distinct latencies < s);
//             rf[n_pad] u16            rank of x's feasible-branch objective;
//             df[n_pad] u16            rf ^ rank of x's infeasible-branch objective (ALPHA);
//             inv[2*n_cfg] u16         rank -> op-local index (op base 2*cfg_off[v]);
//             fast[n_ops]              argmin (L, index), the cost-first fallback.
//   Per call: ref[n_ops], cp[n_ops] int64; bucketing scratch (see llama_ctx).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/llama.h"
#include "../../include/llama_loop.h"

namespace llama {

constexpr int kVec = 8;            // configurations per 128-bit rank vector
constexpr uint16_t kPadRank = 0xFFFF;
constexpr uint16_t kLatRankBias = 0x8000;  // latency ranks are stored as 0x8000 + rank
constexpr uint16_t kLatRankPad = 0xBFFF;   // at pads: above any count of distinct latencies
constexpr int kScoreThreads = 256;
constexpr int kScoreThreadsLog2 = 8;
constexpr int kMaxChunk = 4096;        // table entries staged at a time by the scoring kernel
// Warp tiles: an op whose padded table and distinct latencies fit one warp's
// slice of the scoring kernel's shared memory is scored by single warps, each
// taking 32 * IPT of its invocations, with no block barrier
constexpr int kScoreWarps = kScoreThreads / 32;
constexpr int kWarpSlice = 4608;       // bytes of shared memory per warp in the warp phase
// largest padded table scored by warp tiles: table (4 B per entry, 6 in alpha
// mode) and distinct latencies (at most one 4-byte value per entry) in a slice
__host__ __device__ constexpr int32_t warp_pad_of(int mode) {
    return kWarpSlice / (mode == LLAMA_MODE_ALPHA ? 10 : 8) / kVec * kVec;
}
constexpr int kMaxWaitTries = LLAMA_WAIT_LIMIT_DEFAULT;  // bounded waits (mbarrier, grid barrier)
constexpr int kKeep = 4;               // invocations a counting thread keeps in registers
constexpr int kRound = 4;              // invocations a counting thread takes per round after those
constexpr int kKeepOps = 2;            // ops the layout keeps in registers per thread
constexpr int kMaxDlatSmem = 4096;     // distinct latencies staged per op (else searched in L2)
constexpr int kPfArrays = 20;          // arrays k_bucket prefetches into L2 at its start
constexpr int kCntStride = 32;     // int32 slots between per-op counters: one 128-byte line each
// control words of a call (unsigned long long each)
constexpr int kCtrlInvalid = 0;    // invalid invocations
constexpr int kCtrlCountBarrier = 1;  // grid barrier of k_bucket's counting blocks
constexpr int kCtrlPositions = 2;  // bucket positions laid out
constexpr int kCtrlTiles = 3;      // scoring tiles laid out
constexpr int kCtrlTimeout = 4;    // nonzero: a bounded device wait gave up
constexpr int kCtrlNextTile = 5;   // dynamic tile counter of the scoring kernel
constexpr int kCtrlBarrier = 6;    // grid barrier of k_bucket
constexpr int kCtrlDone = 7;       // CTAs of the scoring kernel that have finished
constexpr int kCtrlNextWarpTile = 8;  // dynamic warp-tile counter of the scoring kernel
constexpr int kCtrlCtaTiles = 9;   // tiles scored by whole CTAs (the warp tiles follow them)
constexpr int kCtrlWords = 10;
// Status of the last completed call, after the control words: {invalid
// invocations, nonzero if a bounded device wait gave up}
constexpr int kStatusWords = 2;
// k_bucket's grid never exceeds this many blocks (per-block layout sums)
constexpr int kMaxBucketBlocks = 4096;
// DAGs up to this size are staged in shared memory for the critical path
constexpr int kCpSmemOps = 512;
constexpr int kCpPackWords = 5120;  // packed DAG words staged in shared memory
constexpr int kCpWarpOps = 128;       // a warp's slice of the critical-path area: ops
constexpr int kCpWarpWords = 384;     // and packed words (<= 384 words implies <= 126 ops)
// k_bucket lays out the buckets without barriers of its own (every counting
// block computes the whole layout) when the ops are at most this many: four
// per thread, their loads all in flight at once; the bucket starts go to the
// block's otherwise unused critical-path staging area
constexpr int kLayoutWholeOps = 4 * 256;
static_assert(kLayoutWholeOps * 4 <= kCpSmemOps * 16 + kCpPackWords * 4, "bucket starts exceed the staging area");

struct DevProblem {
    int32_t n_dags, n_ops, n_hw, mode;
    const int32_t *dag_op_off, *row_ptr, *col;
    const int64_t *slo;
    // [n_dags] per DAG {first op, end of its ops, SLO low 32 bits, SLO high 32
    // bits}: what validating and counting an invocation needs, in one 16-byte load
    const int4 *dag_info;
    const int64_t *cfg_off;
    const int32_t *hw_off;
    const int32_t *lat;
    const int64_t *cost;
    const int32_t *ref_cfg;
    const int32_t *batch, *res, *res_total;
    const int64_t *pad_off;
    const int32_t *seg_pad;
    const uint16_t *lrb;
    const int32_t *dlat, *dlat_n;
    // [n_ops*32] per op with more than 32 distinct latencies, the 32 values a
    // 32-lane search probes first: dlat[pad_off[v] + ((l+1)*dn >> 5) - 1], l < 32
    const int32_t *dpiv;
    // [n_ops*32*32] (null when no op has more than 1,024 configurations) per op
    // and outcome c of a 32-probe first round (c of the dpiv values below the
    // slack), the 32 values a second round probes in the window [lo, hi) that
    // round leaves, lo = c*dn >> 5, hi = ((c+1)*dn >> 5) - 1:
    // dlat[pad_off[v] + lo + ((l+1)*(hi-lo) >> 5) - 1], l < 32, when hi - lo > 32
    const int32_t *dpiv2;
    const uint16_t *rf, *df, *inv;
    const int32_t *fast;
    const int32_t *op_order;  // ops by padded table size, largest first (bucket order)
    int32_t max_npad;  // largest padded op table (entries)
    // ops in bucket order scored by whole CTAs; the rest (padded tables of at
    // most warp_pad entries, the end of the bucket order) by single warps
    int32_t n_cta_ops;
    // ops whose padded tables exceed the distinct latencies the scoring kernel
    // stages: the first n_big_ops of op_order, so their bucket positions come first
    int32_t n_big_ops;
    // 128-byte lines to pull into L2 before scoring (0: off): of each of lrb, rf
    // (and df), all 2*n_pad bytes long, and of dlat (4*n_pad bytes)
    int64_t prefetch_rank_lines, prefetch_dlat_lines;
    // small per-op and per-DAG arrays (and the decode tables when they fit) that
    // the call's dependent load chains touch first: pulled into L2 by every
    // block of k_bucket at its start, in one parallel round
    const char *pf_ptr[kPfArrays];
    int64_t pf_lines[kPfArrays];  // 128-byte lines of each (0: unused)
    const int64_t *ref_gidx;      // [n_ops] cfg_off[v] + ref_cfg[v]
    // [n_ops] per bucket-order position k: {op = op_order[k], vectors of its padded
    // table, its padded offset, its number of distinct latencies}
    const int4 *ord_info;
    const int32_t *ord_cbase;  // [n_ops] cfg_off[op_order[k]] per bucket-order position k
    // Decode tables: for rank r of op v (cost-first: the feasible-branch ranks,
    // dec[cfg_off[v] + r]; alpha: the joint ranks, dec[2*cfg_off[v] + r]), the
    // configuration it stands for: {index | backend << 16, latency, cost low,
    // cost high}; dfast[v]: the same for the op's fastest configuration
    const int4 *dec, *dfast;
    // Staircase method: per op v and backend h, at stair[stair_off[v] + h*(dn+1) + k]
    // for k = 0..dn, the least key among the configurations of segment h whose
    // latency rank is below k (cost-first: feasible-branch ranks, 0xFFFF if none;
    // alpha: that, or the least infeasible-branch rank among those at or above k)
    const uint16_t *stair;
    const int64_t *stair_off;   // H * (n_cfg(v) + 1) keys per op, so feedback can change dn in place
    // encoders only: when set, rebuild just the ops with encode_only[v] != 0
    const uint8_t *encode_only;
    // per DAG, its structure packed contiguously (local op ids): {first op, ops,
    // edges, levels}, reference-configuration indices, successor CSR offsets,
    // successors, ops by height above the sinks, level offsets; empty for a DAG
    // too large for shared memory
    const int32_t *dag_pack;
    const int64_t *dag_pack_off;  // [n_dags+1]
    int64_t *ref;
    int64_t *cp;
    uint64_t *cp_magic;  // floor((2^64-1) / cp[v]), for exact division by cp[v]
    const int64_t *q;  // [n_hw] queueing time per backend (device: set by the host or by Eq. 2)
    int64_t alpha_num, alpha_den;
    // polls of a grid barrier of k_bucket before it gives up (kMaxWaitTries
    // unless a caller lowers it to exercise the give-up path)
    int32_t wait_tries;
    int64_t n_cfg, n_pad;  // configurations, padded table entries (bounds of the checked build)
    unsigned int *check;   // the -DLLAMA_CHECK build's violation bits (LLAMA_CHECK_*)
};

// Bounds checks of the -DLLAMA_CHECK build: a check that fails sets its bit in
// the context's check word (P.check) and the guarded access is skipped -- no
// trap, the call completes and llama_check_word reports it.  In the normal
// build every check is the constant true.
#ifdef LLAMA_CHECK
#define LLAMA_IN_BOUNDS(P, cond, bit) ((cond) ? true : (atomicOr((P).check, (unsigned)(bit)), false))
#else
#define LLAMA_IN_BOUNDS(P, cond, bit) true
#endif

struct BucketScratch {
    int32_t *cnt;             // [n_ops*kCntStride] invocations per op: zero when a call starts
                              // (the scoring kernel clears them once bucketing is done)
    unsigned long long *ctrl; // [kCtrlWords] control words: zero when a call starts; the
                              // scoring kernel's last CTA clears them for the next call
    unsigned long long *status;  // [kStatusWords] written by that CTA: {invalid, timeout}
    int4 *blk;                // [kMaxBucketBlocks] per counting block: bucket positions,
                              // full tiles and tail tiles of its ops (written each call)
    int32_t *op_start;        // [n_ops]     first bucket position of each op
    int32_t *gop;             // [n_inv]     global op of each invocation, -1 if invalid
    int32_t *slot;            // [n_inv]     rank of the invocation inside its op's bucket
    int2 *b_ent;              // [n_inv]     at each bucket position, {invocation, its remaining time
                              //             before queueing, max(0, SLO - elapsed)}: one 8-byte
                              //             store per invocation from the scatter
    int64_t *rbase;           // [n_inv]     target - elapsed time of each invocation
    int4 *tiles;              // [2*max_tiles] scoring tiles: {op, first bucket position, m, lanes_log2},
                              // {padded entries, distinct latencies, padded offset, 0}
    uint16_t *b_cnt;          // [n_inv*n_hw] or null: for the invocation at each bucket position
                              //             whose op's distinct latencies are not staged in shared
                              //             memory, the count of them below its slack per backend
    int64_t n_inv;            // invocations of the call (set by enqueue_schedule)
};

// floor(n / d) for n < 2^62 and d >= 1, given m = floor((2^64 - 1) / d): the high
// half of n*m lies within one of n/d from below (m > 2^64/d - 1, so the error is
// below 2n/2^64 < 1/2), so it is floor(n/d) or one less and one comparison makes it
// exact.  This is division by an invariant integer through multiplication
// (Granlund and Montgomery, PLDI 1994), with the divisor fixed per operation.
__device__ __forceinline__ uint64_t div_invariant(uint64_t n, uint64_t d, uint64_t m) {
    uint64_t q = __umul64hi(n, m);
    if (n - q * d >= d) ++q;
    return q;
}

// Slack of Algorithm 1 through the longest remaining path (Section 4.1):
// floor(ref * R / cp), 0 once the target has passed.  ref, R < 2^31, so
// ref*R < 2^62.
__device__ __forceinline__ int32_t slack_of(int64_t ref, int64_t cp, uint64_t magic, int64_t R) {
    if (R <= 0) return 0;
    return (int32_t)div_invariant((uint64_t)(ref * R), (uint64_t)cp, magic);
}

// Read-only view of a ready context for launchers outside llama_host.cu
// (defined in llama_host.cu).
struct ContextView {
    DevProblem P;
    const int32_t *topo, *lvl_off, *dag_lvl;
    int32_t n_dags, n_ops, n_hw, mode, device, num_sms;
    int32_t method;       // LLAMA_METHOD_SCAN or LLAMA_METHOD_STAIRCASE
    int32_t min_vpl;      // vectors a lane should scan at least (sets lanes per invocation)
    int32_t ipt;          // invocations per scoring thread (1, 2 or 4)
    int32_t stages;       // staging buffers of the scoring kernel (1 or 2)
    int32_t score_grid;   // persistent CTAs of the scoring kernel
    int32_t bucket_max_blocks;  // co-resident blocks of k_bucket (cooperative launch)
    int32_t score_chunk;  // table entries staged per chunk
    int32_t dlat_cap;     // distinct latencies the scoring kernel stages (a multiple of 4)
    size_t score_smem;    // dynamic shared memory of the scoring kernel
    bool need_counts;     // some op may have more distinct latencies than dlat_cap
    int32_t max_ncfg;     // configurations of the largest op
    bool warp_tiles;      // some op is scored by warp tiles (the scoring kernel with the warp phase)
    int64_t direct_max;   // scan-method calls of at most this many invocations skip the bucketing
};
int context_view(llama_ctx *c, ContextView *v);  // LLAMA_OK or the readiness error
int context_fail(llama_ctx *c, int code, const char *msg);
void context_set_launches(llama_ctx *c, int launches);  // what llama_last_launch_count reports

// Kernels (defined in kernels.cu).
__global__ void k_critical_path(DevProblem P, const int32_t *topo, const int32_t *lvl_off,
                                const int32_t *dag_lvl);
__global__ void k_bucket(DevProblem P, int64_t n_inv, const int32_t *dag, const int32_t *op_local,
                         const int64_t *start, int64_t now, BucketScratch S, llama_decision *out,
                         const int32_t *topo, const int32_t *lvl_off, const int32_t *dag_lvl,
                         int32_t min_vpl, int32_t ipt, int32_t n_cp);
// Scoring kernels: objective mode x invocations per thread (1, 2 or 4) x
// staging buffers (k_score: one, tiles claimed dynamically; k_score2: two,
// tiles round-robin) x the warp phase (suffix w: after the whole-CTA tiles,
// the warp tiles of ops whose tables fit a warp's slice).
#define LLAMA_DECLARE_SCORE(name) \
    __global__ void name(DevProblem P, BucketScratch S, llama_decision *out, int32_t chunk, int32_t dl_cap); \
    __global__ void name##w(DevProblem P, BucketScratch S, llama_decision *out, int32_t chunk, int32_t dl_cap);
LLAMA_DECLARE_SCORE(k_score_cf1)
LLAMA_DECLARE_SCORE(k_score_cf2)
LLAMA_DECLARE_SCORE(k_score_cf4)
LLAMA_DECLARE_SCORE(k_score_al1)
LLAMA_DECLARE_SCORE(k_score_al2)
LLAMA_DECLARE_SCORE(k_score_al4)
LLAMA_DECLARE_SCORE(k_score2_cf1)
LLAMA_DECLARE_SCORE(k_score2_cf2)
LLAMA_DECLARE_SCORE(k_score2_cf4)
LLAMA_DECLARE_SCORE(k_score2_al1)
LLAMA_DECLARE_SCORE(k_score2_al2)
LLAMA_DECLARE_SCORE(k_score2_al4)
#undef LLAMA_DECLARE_SCORE
const void *score_kernel(int mode, int ipt, int stages, bool warp);

// Scoring tiles a call may lay out (each op: full tiles plus one tail).
int64_t max_tiles(int64_t n_inv, int32_t n_ops);
// Enqueue the whole scheduling call on stream s: k_bucket, the count pass
// when it runs, k_score (the previous call left the counters and control
// words cleared).  trace (nullable) = LLAMA_TRACE_EVENTS events recorded at
// the phase boundaries.  If a launch fails after the first one went in, the
// counters and control words are cleared by memsets on s (nothing allocated)
// so that the scratch is usable by the next call, and the error is returned.
cudaError_t enqueue_schedule(const ContextView &v, const BucketScratch &S, int64_t n_inv,
                             const int32_t *dag, const int32_t *op_local, const int64_t *start,
                             int64_t now, llama_decision *out, cudaStream_t s,
                             const cudaEvent_t *trace);
__global__ void k_slack(DevProblem P, int64_t n_inv, const int32_t *dag, const int32_t *op_local,
                        const int64_t *start, int64_t now, int32_t *slack_out);
__global__ void k_encode_pad(DevProblem P, uint16_t *lrb, uint16_t *rf, uint16_t *df, int32_t *fast);
__global__ void k_encode_lat(DevProblem P, uint16_t *lrb, int32_t *dlat, int32_t *dlat_n);
__global__ void k_encode_piv(DevProblem P, int32_t *dpiv);
__global__ void k_encode_piv2(DevProblem P, int32_t *dpiv2);
template <int MAXH>
__global__ void k_counts(DevProblem P, BucketScratch S, int32_t dl_cap);
// Kernel launches of one scheduling call (scan method): bucketing, the count
// pass when it runs, scoring.
int schedule_launches(const ContextView &v, const BucketScratch &S, int64_t n_inv);
// Eq. 2: per-backend sums of L(x_i) R(x_i) over decided invocations, then the
// queueing time floor(sum / R_total(lambda)) of every backend.
__global__ void k_queue_sum(DevProblem P, int64_t n, const int32_t *dag, const int32_t *op_local,
                            const llama_decision *dec, unsigned long long *sums);
__global__ void k_queue_finish(DevProblem P, const unsigned long long *sums, int64_t *q_out, int64_t *q_ctx);
// Feedback: observations sorted by global configuration (stable), applied in
// order by exponential smoothing; touched ops flagged for re-encoding.
__global__ void k_feedback_apply(DevProblem P, int64_t n, const int32_t *sorted_g, const int32_t *sorted_obs,
                                 const int32_t *obs_op, const int32_t *obs_lat, const int64_t *obs_cost,
                                 int32_t beta_num, int32_t beta_den, int32_t *lat, int64_t *cost,
                                 uint8_t *touched);
__global__ void k_feedback_keys(DevProblem P, int64_t n, const int32_t *obs_op, const int32_t *obs_cfg,
                                const int32_t *obs_lat, const int64_t *obs_cost, int32_t *keys, int32_t *idx,
                                unsigned long long *rejected);
__global__ void k_refresh_order(DevProblem P, const int32_t *ord_pos, int4 *ord_info);
__global__ void k_gather_u32(int64_t n, const uint32_t *src, const int32_t *idx, uint32_t *dst);
// Eq. 3: per invocation and backend, the least Eq. 1 objective among the op's
// configurations on that backend (a warp per invocation), and the commit keys.
__global__ void k_backend_obj(DevProblem P, int64_t n_inv, const int32_t *dag, const int32_t *op_local,
                              const int64_t *start, int64_t now, int64_t *obj_min);
__global__ void k_commit_keys(DevProblem P, int64_t n, const int32_t *dag, const int32_t *op_local,
                              const llama_decision *dec, const int64_t *obj_min, uint64_t *aff_key,
                              uint32_t *lam_key, int32_t *idx, double *aff_out);
__global__ void k_encode_dec(DevProblem P, int4 *dec, int4 *dfast);
__global__ void k_encode_stair(DevProblem P, uint16_t *stair);
// Staircase method: critical paths of every DAG, then one thread per invocation.
__global__ void k_critical_paths(DevProblem P, const int32_t *topo, const int32_t *lvl_off,
                                 const int32_t *dag_lvl);
__global__ void k_stair(DevProblem P, int64_t n_inv, const int32_t *dag, const int32_t *op_local,
                        const int64_t *start, int64_t now, BucketScratch S, llama_decision *out);
// Small calls of the scan method (at most the context's direct limit of
// invocations): critical paths, then a warp per invocation scanning its op's
// table straight from L2, no bucketing (cost-first and alpha objectives).
__global__ void k_direct_cf(DevProblem P, int64_t n_inv, const int32_t *dag, const int32_t *op_local,
                            const int64_t *start, int64_t now, BucketScratch S, llama_decision *out);
__global__ void k_direct_al(DevProblem P, int64_t n_inv, const int32_t *dag, const int32_t *op_local,
                            const int64_t *start, int64_t now, BucketScratch S, llama_decision *out);
__global__ void k_encode_rank(DevProblem P, int32_t sort_n, uint16_t *rf, uint16_t *df,
                              uint16_t *inv);

// ---------------------------------------------------------------------------
// Serving loop (early speculation and late commit, Section 4.3; priority-based
// commit, Section 4.4): state on the device, one CTA per tick.
// ---------------------------------------------------------------------------
constexpr int kLoopThreads = 1024;  // = LLAMA_LOOP_MAX_ADMIT = LLAMA_LOOP_MAX_COMMIT
static_assert(kLoopThreads == LLAMA_LOOP_MAX_ADMIT && kLoopThreads == LLAMA_LOOP_MAX_COMMIT, "one thread each");

// Page-locked, mapped control words (device writes, host reads; res_read the
// other way round).
struct LoopCtl {
    unsigned long long head;       // requests the device has taken from the ring
    unsigned long long res_count;  // result records published
    unsigned long long res_read;   // records the host has taken (host writes)
    unsigned long long dropped;    // records lost to a full result ring
    unsigned long long ticks;
    unsigned long long inflight;   // admitted and not yet dispatched
};

// Device-resident counters and queue state (one struct in device memory).
struct LoopState {
    unsigned __int128 s_sq[LLAMA_MAX_HW], s_cq[LLAMA_MAX_HW];  // exact sums of L(x) R(x) per queue
    long long sq_head[LLAMA_MAX_HW], sq_tail[LLAMA_MAX_HW], cq_head[LLAMA_MAX_HW], cq_tail[LLAMA_MAX_HW];
    long long head, ticks, admitted, rejected, committed, dispatched, res_count, dropped;
    int32_t free_top;  // free slots on the stack
};

struct LoopDev {
    LoopState *st;
    LoopCtl *ctl;                       // device view of the mapped control words
    const llama_loop_request *ring;     // device view of the mapped request ring
    llama_loop_result *res;             // device view of the mapped result ring
    int64_t ring_mask, res_cap;
    int32_t *free_stack;                // [slots]
    int64_t *slot_id, *slot_start;      // [slots]
    int32_t *slot_dag, *slot_opl;       // [slots]
    unsigned long long *slot_lr_spec, *slot_lr_commit;  // [slots] L(x) R(x) of each decision
    int32_t *sq;                        // [n_hw][slots] speculative queues (rings of slot ids)
    int32_t *cq;                        // [n_hw][cq_stride] commit queues
    int64_t *q;                         // [LLAMA_MAX_HW] the tick's queueing time (P.q points here)
    // Eq. 3's per-backend minima per op, backend and count of distinct latencies
    // below the slack (k_encode_objmin; the staircase tables' indexing)
    int64_t *objmin;
    int32_t slots, cq_stride, max_admit;
    int32_t cq_cap[LLAMA_MAX_HW];
};

struct LoopTickArgs {
    int64_t now, limit;                 // the tick's time; requests submitted before it (ring tail)
    int32_t dispatch[LLAMA_MAX_HW];     // invocations each backend took from its commit queue
};

// Enqueue one tick on s (P.q must be L.q).
cudaError_t enqueue_loop_tick(const DevProblem &P, const LoopDev &L, const LoopTickArgs &a, cudaStream_t s);
// Critical paths of every DAG (a1), on s.
cudaError_t enqueue_critical_paths(const ContextView &v, cudaStream_t s);
int context_ensure_stair(llama_ctx *c);  // staircase tables for the current profiles
// Eq. 3's minima tables of the current profiles into objmin (as many elements
// as the staircase tables, H * (n_cfg + n_ops)), on s.
cudaError_t enqueue_encode_objmin(const ContextView &v, int64_t *objmin, cudaStream_t s);

}  // namespace llama
