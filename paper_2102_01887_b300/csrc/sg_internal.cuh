// Internal interfaces of the surrogate's CUDA code (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace sgk {

// Arguments of the fused selection epilogue (see mlp_layer_select).
struct SelectArgs {
    const float *w4 = nullptr;        // [256] row 0 of the last layer
    const float *b4 = nullptr;        // its bias (device)
    // per pair: (invocation, op-local configuration index, profiled latency,
    // slack of the invocation on the configuration's backend)
    const int4 *pair_sel = nullptr;
    const int64_t *pair_cost = nullptr;  // per pair: profiled cost per invocation
    float margin = 0.f;               // added to the predicted log factor before selection
    unsigned long long *best = nullptr;  // [n_inv] best key so far
    int32_t *lhat = nullptr;             // [pairs] predicted latency
    int64_t *chat = nullptr;             // [pairs] predicted cost
};

// C = A . B^T on the tensor cores; see llama_gemm_bf16 for shapes and limits.
int gemm(const void *a, const void *b, const float *bias, void *c16, float *c32, int64_t m, int n, int k,
         int flags, cudaStream_t s);
// The same product into FP32 c32 [m x n] (no bias, no activation) with K split
// over `splits` CTAs per output tile (a power of two dividing k / 64): each
// writes its partial product to part (splits * m * n floats, at most part_bytes),
// then one pass sums the partials in a fixed order, so the result does not
// depend on scheduling.  For products with few output tiles and a long K
// (weight gradients: K = the batch).
constexpr int kMinSplitBlocks = 8;  // K blocks of 64 per split at least
int splits_for(int64_t m, int n, int k, int sms);
int gemm_split_k(const void *a, const void *b, float *c32, int64_t m, int n, int k, int splits, float *part,
                 size_t part_bytes, cudaStream_t s);
struct llama_mlp_view {
    const float *params;       // FP32 master parameters (flat layout above)
    const void *w16[4];        // BF16 W1..W4 [out x in]
    int device;
    int64_t version;           // changes whenever the weights change
};

// The pair layers of the scheduling path on the persistent kernel (weights kept
// in shared memory, double-buffered accumulators), w [256 x 256] BF16.
// Layer 2 with the first layer built in the kernel: row r of tile t (128 rows)
// has h1 = ReLU(a_cfg[tile_info[t].x + r] + b_inv[tile_info[t].y]) (a_cfg BF16
// [n_cfg x 256], b_inv FP32 [n_inv x 256]), c16 [m x 256] = ReLU(h1 . w^T + bias)
// in BF16, m a multiple of 128.
int mlp_layer_first(const void *a_cfg, int64_t n_cfg, const float *b_inv, const int2 *tile_info, const void *w,
                    const float *bias, void *c16, int64_t m, cudaStream_t s);
// Layer 3 over a [m x 256] BF16 with the fused last layer and selection; rows
// whose selection record has a negative invocation are skipped.
int mlp_layer_select(const void *a, const void *w, const float *bias, int64_t m, const SelectArgs &sel,
                     cudaStream_t s);
// The device word that bounded waits of the GEMM set when they give up.
int *error_word();

constexpr int kIn = 64, kHid = 256, kOut = 64;  // network widths (inputs and outputs padded)
constexpr int kTileRows = 128;                   // rows per tile of the pair layers
// flat parameter layout: W1[256x64] b1 W2[256x256] b2 W3[256x256] b3 W4[64x256] b4[64]
constexpr int64_t kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid,
                  kOffB2 = kOffW2 + kHid * kHid, kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid * kHid,
                  kOffW4 = kOffB3 + kHid, kOffB4 = kOffW4 + kOut * kHid, kParams = kOffB4 + kOut;

}  // namespace sgk

struct llama_mlp;
namespace sgk {
llama_mlp_view mlp_view(const llama_mlp *m);
}  // namespace sgk
