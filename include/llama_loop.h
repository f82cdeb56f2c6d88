/*
 * llama_loop.h -- device-resident serving loop of the scheduling step:
 * early speculation and late commit (Section 4.3) with priority-based commit
 * (Section 4.4), every piece of in-flight state held on the GPU.
 *
 * Requests (pending operation invocations) are written by the host into a
 * page-locked ring that the device reads in place.  Each tick is one kernel
 * launch that, on the device:
 *
 *   1. dispatch: removes dispatch[lambda] invocations from the head of each
 *      commit queue CQ[lambda] (the backend started them; the caller, which
 *      runs the backends, reports how many) and frees their slots;
 *   2. admit: takes requests from the ring in arrival order while slots are
 *      free (the slot count is the loop's device-memory budget), at most
 *      max_admit per tick and none submitted after the tick was launched;
 *   3. speculate (early speculation): gives each admitted invocation its
 *      slack (Algorithm 1) under the queueing time of every backend at the
 *      tick's start, Q[lambda] = floor((S_SQ + S_CQ) / R_total(lambda)) where
 *      S_SQ, S_CQ are the exact sums of L(x_i) R(x_i) over the invocations
 *      in SQ[lambda] and CQ[lambda] (Eq. 2, both queues), selects its
 *      configuration x (Eq. 1) and appends it to the speculative queue
 *      SQ[lambda(x)], in arrival order;
 *   4. commit (late commit): re-scores the first cq_cap[lambda] entries of
 *      every SQ[lambda] -- Algorithm 1 and Eq. 1 again, at the tick's time,
 *      under the queueing time after step 3 (which counts the speculative
 *      queues, the invocations behind each candidate included) -- and
 *      commits them into the commit queue of their re-scored backend
 *      lambda', in the priority order of Section 4.4: by lambda', then by
 *      descending affinity (Eq. 3: the least Eq. 1 objective of the
 *      invocation's operation on the other backends over the least on
 *      lambda'; +inf when the latter is 0, 1.0 when both are), then by
 *      candidate order (source backend, then queue position), while
 *      CQ[lambda'] has room.  A candidate that finds no room stays in its
 *      speculative queue, in order, with its speculative decision.
 *
 * Every admitted request gives one result record (speculated, or rejected
 * when invalid), and one more when it is committed; records are written to a
 * page-locked ring the host polls.  Decisions are computed with the staircase
 * tables (exactly the configurations Eq. 1 selects over all configurations),
 * Eq. 3's per-backend minima with the context's alpha.  Everything a tick does
 * is deterministic: the same submissions, tick times and dispatch counts give
 * the same records.
 *
 * The paper has no counterpart for the ring, the slot budget or the
 * dispatch counts: they are how a serving process feeds this loop.
 */
#ifndef LLAMA_LOOP_H
#define LLAMA_LOOP_H

#include <stdint.h>

#include "llama.h"

#ifdef __cplusplus
extern "C" {
#endif

#define LLAMA_LOOP_MAX_ADMIT 1024  /* requests a tick admits at most */
#define LLAMA_LOOP_MAX_COMMIT 1024 /* sum of the commit-queue capacities */

typedef struct llama_loop_opts {
    int32_t slots;      /* invocations in flight on the device (admitted, not yet dispatched),
                           1..1<<22: the loop's device-memory budget */
    int32_t ring;       /* request ring capacity, a power of two, 2..1<<24 */
    int32_t results;    /* result ring capacity, a power of two, 2..1<<24 */
    int32_t max_admit;  /* requests admitted per tick, 1..LLAMA_LOOP_MAX_ADMIT */
    int32_t cq_cap[LLAMA_MAX_HW]; /* commit-queue capacity per backend, >= 1, summing to at
                                     most LLAMA_LOOP_MAX_COMMIT */
} llama_loop_opts;

typedef struct llama_loop_request {
    int64_t id;        /* the caller's identifier */
    int32_t dag;       /* pipeline of the invocation */
    int32_t op_local;  /* operation within it */
    int64_t start_us;  /* start of the pipeline instance (<= the admitting tick's time) */
} llama_loop_request;

#define LLAMA_LOOP_SPECULATED 1 /* admitted: speculative decision */
#define LLAMA_LOOP_COMMITTED 2  /* committed: the decision it runs with */
#define LLAMA_LOOP_REJECTED 3   /* invalid invocation: not admitted, cfg = -1 */

typedef struct llama_loop_result {
    int64_t id;
    int32_t kind;            /* LLAMA_LOOP_* */
    int32_t tick;            /* tick that produced the record (0-based) */
    llama_decision decision;
    int32_t backend;         /* lambda of the decision's configuration, -1 if rejected */
    int32_t pad;
} llama_loop_result;

typedef struct llama_loop_state {
    int64_t ticks, submitted, admitted, rejected, committed, dispatched, results;
    int64_t results_dropped;           /* records lost to a full result ring (poll faster) */
    int32_t free_slots;
    int32_t sq_len[LLAMA_MAX_HW], cq_len[LLAMA_MAX_HW];
    int64_t q_us[LLAMA_MAX_HW];        /* Eq. 2 over both queues, now */
} llama_loop_state;

typedef struct llama_loop llama_loop;

/* A loop over a ready context: DAGs and profiles set, with batch, res and
 * res_total (Eq. 2 and Eq. 3 need B(x), R(x) and R_total).  Builds the
 * staircase tables for the current profiles (if the context has none), the
 * loop's tables of Eq. 3's per-backend minima (per op, backend and count of
 * distinct latencies below the slack: 8 B per configuration and backend) and
 * the critical paths.  Call
 * llama_loop_refresh after the context's tables change (feedback); a new
 * llama_set_profiles needs a new loop.  The loop owns a CUDA stream, device
 * state sized by opts, and two page-locked rings.  Errors: EINVAL, ENOTREADY,
 * ENOMEM, ECUDA. */
int llama_loop_create(llama_ctx *ctx, const llama_loop_opts *opts, llama_loop **out);
void llama_loop_destroy(llama_loop *loop);

/* Write n requests into the ring (host only; not thread-safe against
 * another submit; safe beside the driver thread).  All or nothing: EINVAL for bad arguments, LLAMA_EAGAIN
 * (-6) when the ring lacks room for all n. */
int llama_loop_submit(llama_loop *loop, const llama_loop_request *req, int64_t n);

/* Enqueue one tick at time now_us on the loop's stream (returns without
 * waiting).  dispatch (host, n_hw entries, nullable = none): invocations each
 * backend took from the head of its commit queue since the last tick.  The
 * tick admits only requests submitted before this call.  Errors: EINVAL,
 * ECUDA. */
int llama_loop_tick(llama_loop *loop, int64_t now_us, const int32_t *dispatch);

/* Run the ticks on a native host thread of the library (the "driver"):
 * whenever fewer than ticks_in_flight ticks are queued on the loop's stream,
 * it enqueues one at the steady clock's time (now_us at the start, plus the
 * microseconds since), with the same dispatch counts every tick (host,
 * n_hw entries, nullable = none; INT32_MAX dispatches each commit queue whole,
 * for backends that keep up).  The driver spins on the control words (it
 * keeps one host core busy) while ticks are queued; once the ring is empty and
 * nothing is in flight it spins a while longer, then sleeps 20 us between polls.  The caller keeps submitting and
 * polling; llama_loop_tick is refused while the driver runs.  Ticks are then
 * timed by the clock, so their records are not reproducible run to run (each
 * tick still does exactly what llama_loop_tick would).  Errors: EINVAL. */
int llama_loop_start(llama_loop *loop, int64_t now_us, int32_t ticks_in_flight, const int32_t *dispatch);

/* Stop the driver thread and wait for its ticks.  Errors: ECUDA (a tick
 * launch failed; the driver stopped then). */
int llama_loop_stop(llama_loop *loop);

/* Copy up to max_out result records, oldest first, into out (host); their
 * number in *n_out.  Never waits for the GPU. */
int llama_loop_poll(llama_loop *loop, llama_loop_result *out, int64_t max_out, int64_t *n_out);

/* A native arrival process (no counterpart in the paper): on the calling host
 * thread, submit req[k] (whose ids must be id0 + k) once arrive_ns[k]
 * (non-decreasing, nanoseconds after this call starts) has passed -- as many
 * as the ring takes, the rest at the next pass -- and poll the records, until
 * every request's speculative and commit records are seen or timeout_ns has
 * passed; spec_ns[k] and commit_ns[k] (host, n each) receive when each record
 * was seen (ns after the start; -1 if not seen; a rejected request gets both
 * at its rejection).  The driver thread (llama_loop_start) must run the ticks.
 * Spins on one host core; nothing is allocated on the device.  Errors:
 * EINVAL, and any error of llama_loop_submit or llama_loop_poll. */
int llama_loop_run_arrivals(llama_loop *loop, const llama_loop_request *req, const int64_t *arrive_ns, int64_t n,
                            int64_t id0, int64_t timeout_ns, int64_t *spec_ns, int64_t *commit_ns);

/* Ticks completed so far (read from the page-locked control words the last
 * tick published; never waits), or -1 for a null loop. */
int64_t llama_loop_ticks_done(llama_loop *loop);

/* Wait until every enqueued tick has completed.  Errors: ECUDA. */
int llama_loop_sync(llama_loop *loop);

/* The loop's counters and queues after the ticks enqueued so far (waits for
 * them).  Errors: EINVAL, ECUDA. */
int llama_loop_state_get(llama_loop *loop, llama_loop_state *st);

/* Rebuild the loop's tables and critical paths from the context's current
 * profiles (after llama_feedback); waits for the loop's stream.  Errors:
 * ENOMEM, ECUDA. */
int llama_loop_refresh(llama_loop *loop);

#ifdef __cplusplus
}
#endif

#endif /* LLAMA_LOOP_H */
