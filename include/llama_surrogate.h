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

#ifdef __cplusplus
}
#endif

#endif /* LLAMA_SURROGATE_H */
