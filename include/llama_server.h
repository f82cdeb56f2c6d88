/*
 * llama_server.h -- C ABI of the serving loop around the scheduling step.
 *
 * Invocations arrive one by one (a pipeline's operation becomes ready) and
 * must each get a decision quickly (Section 4: the Configurator decides as
 * invocations become ready).  The server batches them continuously: whenever
 * one of its slots is free, every queued request (up to max_batch) is copied
 * to the GPU and scheduled on that slot's stream with that slot's workspace,
 * while earlier batches are still running on theirs; results are collected as
 * their batches complete.  Slots are sized by a device-memory budget, and the
 * queue is bounded (admission control).  Everything here runs on the host
 * thread that calls poll: no device-side waiting.
 *
 * Each request carries the time it is decided at (now_us); a batch schedules
 * every request against its own now_us, so a request's decision is the same
 * whichever batch it lands in, and the same as scheduling it alone.
 */
#ifndef LLAMA_SERVER_H
#define LLAMA_SERVER_H

#include <stdint.h>

#include "llama.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct llama_request {
    int64_t id;        /* caller's identifier, returned with the result */
    int32_t dag;       /* pipeline (DAG) of the invocation */
    int32_t op_local;  /* operation within it */
    int64_t start_us;  /* start of the pipeline instance */
    int64_t now_us;    /* the time the decision is taken at */
} llama_request;

typedef struct llama_result {
    int64_t id;
    llama_decision decision;
    int64_t submit_ns;  /* host steady clock at submission */
    int64_t done_ns;    /* host steady clock when the result was collected */
} llama_result;

typedef struct llama_server_opts {
    int32_t slots;          /* concurrent batches; 0 = as many as the budget allows (1..64) */
    int32_t max_batch;      /* requests per batch, 1 .. 1<<20 */
    int64_t memory_budget;  /* device bytes for the slots' buffers and workspaces (slots = 0) */
    int64_t max_queue;      /* queued requests beyond which submit refuses (0 = 1<<24) */
} llama_server_opts;

typedef struct llama_server_stats {
    int64_t submitted, completed, refused, batches;
    int32_t slots;
    int32_t max_in_flight;    /* most batches in flight on the GPU at one launch */
    int64_t overlapped;       /* batches whose device interval overlapped another batch's */
    int64_t queue_peak;
    double device_busy_ms;    /* union of the batches' device intervals */
    double device_span_ms;    /* first batch start to last batch end */
} llama_server_stats;

typedef struct llama_server llama_server;

/* A server over a ready context (DAGs and profiles set).  Errors: EINVAL,
 * ENOTREADY, ENOMEM, ECUDA. */
int llama_server_create(llama_ctx *ctx, const llama_server_opts *opts, llama_server **out);
void llama_server_destroy(llama_server *srv);

/* Queue n requests (thread-safe).  All or nothing: EINVAL (null or n < 0) or
 * LLAMA_EAGAIN when the queue would exceed max_queue (the requests are
 * refused and counted). */
#define LLAMA_EAGAIN (-6)
int llama_server_submit(llama_server *srv, const llama_request *req, int64_t n);

/* Launch queued requests into free slots and collect completed batches
 * (never blocks on the GPU): up to max_out results into out, their number in
 * *n_out; results not yet taken stay for the next call.  Errors: EINVAL,
 * ECUDA (a batch failed: the server stops). */
int llama_server_poll(llama_server *srv, llama_result *out, int64_t max_out, int64_t *n_out);

/* Poll until every submitted request has been returned or timeout_ms passes
 * (then ETIMEOUT); results as for poll. */
int llama_server_drain(llama_server *srv, llama_result *out, int64_t max_out, int64_t *n_out,
                       int64_t timeout_ms);

int llama_server_stats_get(llama_server *srv, llama_server_stats *st);

#ifdef __cplusplus
}
#endif

#endif /* LLAMA_SERVER_H */
