// Internal interfaces of the surrogate's CUDA code (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace llama_sg {

// C = A . B^T on the tensor cores; see llama_gemm_bf16 for shapes and limits.
int gemm(const void *a, const void *b, const float *bias, void *c16, float *c32, int64_t m, int n, int k,
         int flags, cudaStream_t s);
// The device word that bounded waits of the GEMM set when they give up.
int *error_word();

constexpr int kIn = 64, kHid = 256, kOut = 64;  // network widths (inputs and outputs padded)
// flat parameter layout: W1[256x64] b1 W2[256x256] b2 W3[256x256] b3 W4[64x256] b4[64]
constexpr int64_t kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid,
                  kOffB2 = kOffW2 + kHid * kHid, kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid * kHid,
                  kOffW4 = kOffB3 + kHid, kOffB4 = kOffW4 + kOut * kHid, kParams = kOffB4 + kOut;

}  // namespace llama_sg
