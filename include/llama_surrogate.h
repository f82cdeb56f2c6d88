/*
 * llama_surrogate.h -- C ABI of the learned latency surrogate of the
 * B300-native Llama scheduling step.
 *
 * The paper profiles every configuration offline and treats a table of
 * latencies as fixed (Section 3.2), while noting that an operation's latency
 * varies with the content of the frames it processes (Section 2, Fig. 3).  The
 * surrogate is a small MLP (BF16 weights and activations, FP32 accumulation)
 * that predicts an operation's latency from the configuration's knob and
 * hardware features and the invocation's content features; the profile table
 * stays the fallback and the reference its decisions are judged against.  The
 * paper has no counterpart of this network: it is an extension, trained on
 * the GPU by the kernels declared here.
 *
 * Conventions: matrices are row-major; BF16 is the IEEE-754 binary32 upper
 * half (round to nearest even); pointers are device memory; calls are
 * enqueued on `stream` (a cudaStream_t, NULL = legacy default stream) and do
 * not wait.  Status codes are those of llama.h.
 */
#ifndef LLAMA_SURROGATE_H
#define LLAMA_SURROGATE_H

#include <stdint.h>

#include "llama.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Epilogue flags of llama_gemm_bf16. */
#define LLAMA_GEMM_RELU 1 /* C = max(C, 0) after the bias */

/* C[m x n] = A[m x k] . B[n x k]^T (+ bias[n]) (ReLU if LLAMA_GEMM_RELU) on the
 * tensor cores: A and B BF16, row-major (both K-major), accumulation in FP32;
 * the result is written as BF16 to c_bf16 and/or FP32 to c_f32 (either may be
 * NULL, not both), row-major with leading dimension n.  bias (FP32, n) may be
 * NULL.  Limits: k a multiple of 64; n = 64 or a multiple of 128; all pointers
 * 16-byte aligned.  Errors: EINVAL (shape, alignment, or a tensor map the
 * driver rejects), ECUDA (launch), ENOMEM.  A device-side wait that gives up
 * is reported later by llama_gemm_error. */
int llama_gemm_bf16(const void *a, const void *b, const float *bias, void *c_bf16, float *c_f32,
                    int64_t m, int32_t n, int32_t k, int32_t flags, void *stream);

/* LLAMA_ETIMEOUT if any GEMM since the last clearing call had a bounded
 * device wait give up (its outputs are then invalid), else LLAMA_OK.
 * Synchronous (reads one device word); clear != 0 resets the flag. */
int llama_gemm_error(int32_t clear);

/* The network: LLAMA_MLP_INPUTS inputs (48 features in use: 32 describing the
 * configuration and its operation, 16 the invocation's frame content; the
 * rest zero), three hidden layers of 256 with ReLU, LLAMA_MLP_OUTPUTS outputs
 * of which the first two are read: y0 = log(latency / profiled latency) and
 * y1 = branch fan-out.  Loss: the batch mean of (y0 - t0)^2 / 2 +
 * w_fan (y1 - t1)^2 / 2.  Parameters travel as LLAMA_MLP_PARAMS FP32 values in
 * the order W1[256x64], b1[256], W2[256x256], b2, W3[256x256], b3, W4[64x256],
 * b4[64] (row-major, W[out x in]).  Products run on the tensor cores in BF16
 * with FP32 accumulation; the FP32 parameters are the master copy. */
#define LLAMA_MLP_INPUTS 64
#define LLAMA_MLP_OUTPUTS 64
#define LLAMA_MLP_PARAMS 164672

typedef struct llama_mlp llama_mlp;

/* A network on `device` with activation buffers for batches of up to
 * max_batch rows (128 .. 2^26), parameters zero.  Errors: EINVAL, ENOMEM, ECUDA. */
int llama_mlp_create(llama_mlp **out, int32_t device, int64_t max_batch);
void llama_mlp_destroy(llama_mlp *net);

/* Copy LLAMA_MLP_PARAMS FP32 values from / to host memory (blocking).  Setting
 * the parameters also resets the optimizer state. */
int llama_mlp_set_params(llama_mlp *net, const float *params);
int llama_mlp_get_params(llama_mlp *net, float *params);

/* Outputs y0, y1 of n rows of x (BF16 [n x 64], device, 16-byte aligned) into
 * y (FP32 [n x 2], device).  1 <= n <= max_batch. */
int llama_mlp_forward(llama_mlp *net, const void *x, int64_t n, float *y, void *stream);

/* Gradient of the mean loss over n rows (a multiple of 128) of x with targets
 * t (FP32 [n x 2], device): written to grads (FP32 [LLAMA_MLP_PARAMS], device)
 * unless NULL; the loss is written to *loss (device) unless NULL. */
int llama_mlp_gradients(llama_mlp *net, const void *x, const float *t, int64_t n, float w_fan,
                        float *grads, float *loss, void *stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) at
 * learning rate lr on the gradient of that batch; *loss (device) gets the
 * batch loss before the step unless NULL. */
int llama_mlp_train_step(llama_mlp *net, const void *x, const float *t, int64_t n, float w_fan, float lr,
                         float *loss, void *stream);

/* An epoch of Adam steps without a host round trip per step: for b <
 * n_batches, the rows perm[b*batch .. (b+1)*batch) of x (BF16 [n_rows x 64],
 * device, 16-byte aligned) and t (FP32 [n_rows x 2], device) are gathered on
 * the device into the network's own batch buffers, then llama_mlp_train_step's
 * step is taken on them.  batch: a multiple of 128, at most max_batch; perm
 * (int32 [n_batches*batch], device): row indices, an index outside
 * 0..n_rows-1 giving a zero row.  The batches' losses (each before its step)
 * are added to *loss_sum (device) unless NULL.  The result equals the same
 * batches taken one llama_mlp_train_step at a time.  Errors: EINVAL, ECUDA. */
int llama_mlp_train_epoch(llama_mlp *net, const void *x, const float *t, int64_t n_rows, const int32_t *perm,
                          int64_t n_batches, int64_t batch, float w_fan, float lr, float *loss_sum, void *stream);

/* One-line description of the network's last failure. */
const char *llama_mlp_last_error(llama_mlp *net);

/* Scheduling with the surrogate: the decisions of llama_schedule (cost-first,
 * Algorithm 1's slack on the profiled reference latencies, Eq. 1's selection),
 * with every configuration's latency and cost replaced by the profiled value
 * times e^y0, y0 the network's prediction for (configuration, invocation
 * content).  The context `ctx` supplies the DAGs, SLOs, queueing times and
 * profile tables; `net` the weights (not copied: later training is seen).  A
 * prediction that is not finite falls back to the profiled value.  Decisions
 * report the predicted latency and cost of the chosen configuration and the
 * slack of its backend; FEASIBLE means predicted latency < slack.  At most
 * max_inv invocations and max_pairs (invocation, configuration) pairs per
 * call.  The scratch of a call is allocated here -- for max_inv invocations,
 * and pair rows (whole 128-row tiles per invocation, about 550 B per row) for
 * max_pairs pairs and the padding of up to 4,096 invocations -- so a call
 * allocates nothing but, once per profile, layer 1's configuration part, and,
 * when it needs more pair rows than any call before, their growth (to twice the
 * rows held at least).  Errors: EINVAL, ENOMEM, ECUDA. */
typedef struct llama_sg llama_sg;
int llama_sg_create(llama_sg **out, llama_ctx *ctx, llama_mlp *net, int64_t max_inv, int64_t max_pairs);
void llama_sg_destroy(llama_sg *sg);

/* cfg_x: BF16 [n_cfg x 64] device, row g = global configuration g, features
 * of the configuration in columns 0..31, zeros elsewhere; inv_x: BF16
 * [n_inv x 64] device, row i = invocation i, content features in columns
 * 32..47, zeros elsewhere.  dag, op_local, start_us, out: device, as in
 * llama_schedule_async.  Blocks until the number of pairs is known (one
 * device-to-host read), then enqueues the rest on `stream`. */
int llama_sg_schedule(llama_sg *sg, const void *cfg_x, const void *inv_x, int64_t n_inv, const int32_t *dag,
                      const int32_t *op_local, const int64_t *start_us, int64_t now_us, llama_decision *out,
                      void *stream);

/* Layer 1's configuration part (cfg_x times W1, every configuration) is
 * computed by the first call and kept while later calls pass the same cfg_x
 * pointer, the network's weights are unchanged (llama_mlp_set_params and
 * llama_mlp_train_step change them) and the context's profiles are the same
 * buffers; calls that reuse it must be ordered after the call that computed it
 * (one stream, or an event).  After changing cfg_x's contents in place, call
 * llama_sg_invalidate.  No counterpart in the paper.  Errors: EINVAL. */
int llama_sg_invalidate(llama_sg *sg);

/* A native arrival process for the surrogate's path (no counterpart in the
 * paper), on the calling host thread: continuous batching -- each call of
 * llama_sg_schedule (at time now_us plus the microseconds since this call
 * started) takes every request k whose arrive_ns[k] (non-decreasing, ns after
 * the start) has passed, at most max_batch, then copies the decisions to
 * host_out (page-locked, max_batch entries) on `stream` and waits for them;
 * done_ns[k] (host, n) receives when request k's decision was on the host.
 * inv_x, dag, op_local, start_us: device, per request (inv_x rows as for
 * llama_sg_schedule); out: device, max_batch entries.  Errors: EINVAL, ECUDA,
 * and those of llama_sg_schedule. */
int llama_sg_run_arrivals(llama_sg *sg, const void *cfg_x, const void *inv_x, const int32_t *dag,
                          const int32_t *op_local, const int64_t *start_us, int64_t n, const int64_t *arrive_ns,
                          int64_t now_us, int64_t max_batch, llama_decision *out, llama_decision *host_out,
                          void *stream, int64_t *done_ns);

/* Safety margin in log units (0 .. 1, default 0): the selection uses
 * e^(y0 + margin) times the profiled latency and cost, an upper quantile of the
 * prediction when margin is about the model's error.  Selecting the cheapest
 * configuration among noisy predictions favours underestimated ones; the
 * margin offsets that.  Errors: EINVAL. */
int llama_sg_set_margin(llama_sg *sg, float margin);

/* Pairs of the last call (sum over valid invocations of their operation's
 * configurations), -1 on a null handle. */
int64_t llama_sg_last_pairs(llama_sg *sg);

/* Per pair of the last call (pairs of invocation i at pair_off[i] ..
 * pair_off[i+1], in configuration order): predicted latency (int32) and cost
 * (int64); pair_off has n_inv + 1 entries.  Device pointers, each nullable;
 * enqueued on `stream`.  n_inv must be the last call's.  Errors: EINVAL. */
int llama_sg_predictions(llama_sg *sg, int32_t *lhat, int64_t *chat, int64_t *pair_off, int64_t n_inv,
                         void *stream);

const char *llama_sg_last_error(llama_sg *sg);

#ifdef __cplusplus
}
#endif

#endif /* LLAMA_SURROGATE_H */
