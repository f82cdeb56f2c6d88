// The latency surrogate's network on the GPU: forward pass, gradients of the
// mean loss, and Adam training steps, every matrix product on the tensor cores
// (sg_gemm.cu), the rest in small elementwise kernels here.
//
// Network: 64 inputs (48 features, zero padding) -> 256 -> 256 -> 256 (ReLU)
// -> 64 outputs of which the first two are read: y0 = log(latency / profiled
// latency), y1 = branch fan-out.  Loss: mean over the batch of
// (y0 - t0)^2 / 2 + w_fan (y1 - t1)^2 / 2.  Weights are kept in FP32 (the
// master copy Adam updates) and as BF16 for the products, both as W (forward:
// h W^T) and W^T (backward: dz W); activations are BF16, accumulation FP32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>

#include "llama_surrogate.h"
#include "sg_internal.cuh"

using namespace sgk;

namespace {

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaError_t alloc(size_t n) {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        if (n == 0) return cudaSuccess;
        const cudaError_t e = cudaMalloc(&p, n);
        if (e == cudaSuccess) bytes = n;
        return e;
    }
    ~Buf() {
        if (p) cudaFree(p);
    }
    template <class T>
    T *as() const { return static_cast<T *>(p); }
};

using bf16 = __nv_bfloat16;

// dst [cols x rows] = src [rows x cols]^T (BF16; cols a multiple of 64), in
// 64 x 64 tiles: pairs of elements loaded and stored as 4-byte words, so a
// warp reads and writes 128 contiguous bytes.
constexpr int kTT = 64;  // tile side of the transposes
__global__ void k_transpose(const bf16 *__restrict__ src, bf16 *__restrict__ dst, int64_t rows, int cols) {
    __shared__ bf16 tile[kTT][kTT + 2];
    const int64_t r0 = blockIdx.y * (int64_t)kTT;
    const int c0 = blockIdx.x * kTT, tx = threadIdx.x;
    for (int j = threadIdx.y; j < kTT; j += blockDim.y) {
        const int64_t r = r0 + j;
        const __nv_bfloat162 v = r < rows ? *reinterpret_cast<const __nv_bfloat162 *>(src + r * cols + c0 + 2 * tx)
                                          : __floats2bfloat162_rn(0.f, 0.f);
        tile[j][2 * tx] = v.x;
        tile[j][2 * tx + 1] = v.y;
    }
    __syncthreads();
    const int64_t r = r0 + 2 * tx;
    for (int j = threadIdx.y; j < kTT; j += blockDim.y) {
        bf16 *d = dst + (int64_t)(c0 + j) * rows + r;
        if (r + 1 < rows) {
            __nv_bfloat162 v;
            v.x = tile[2 * tx][j];
            v.y = tile[2 * tx + 1][j];
            if ((rows & 1) == 0) *reinterpret_cast<__nv_bfloat162 *>(d) = v;  // 4-byte aligned
            else d[0] = v.x, d[1] = v.y;
        } else if (r < rows) {
            d[0] = tile[2 * tx][j];
        }
    }
}

// Loss and its gradient with respect to the outputs (rows of 64, two read).
__global__ void k_loss_grad(const float *__restrict__ y, const float *__restrict__ t, int64_t n, float w_fan,
                            bf16 *__restrict__ dy, float *__restrict__ db4, float *__restrict__ loss) {
    __shared__ float red[3][8];
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float l = 0.f, g0 = 0.f, g1 = 0.f;
    if (r < n) {
        const float e0 = y[r * kOut] - t[2 * r], e1 = y[r * kOut + 1] - t[2 * r + 1];
        const float inv = 1.f / (float)n;
        l = 0.5f * (e0 * e0 + w_fan * e1 * e1) * inv;
        g0 = e0 * inv;
        g1 = w_fan * e1 * inv;
        // columns 2..kOut-1 of dy stay zero (cleared when the network is created)
        *reinterpret_cast<__nv_bfloat162 *>(dy + r * kOut) = __floats2bfloat162_rn(g0, g1);
    }
    for (int o = 16; o > 0; o >>= 1) {
        l += __shfl_xor_sync(0xffffffffu, l, o);
        g0 += __shfl_xor_sync(0xffffffffu, g0, o);
        g1 += __shfl_xor_sync(0xffffffffu, g1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = l;
        red[1][threadIdx.x >> 5] = g0;
        red[2][threadIdx.x >> 5] = g1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s0 += red[0][w], s1 += red[1][w], s2 += red[2][w];
        if (loss) atomicAdd(loss, s0);
        atomicAdd(db4, s1);
        atomicAdd(db4 + 1, s2);
    }
}

// Through a ReLU: dz = dh where the layer's output h was positive; dz is
// written row-major and transposed, and its column sums (the bias gradient)
// are accumulated.  64 x 64 tiles of the kHid columns, pairs of elements per
// thread (8-byte loads of dh, 4-byte loads and stores of BF16).
__global__ void k_relu_back(const float *__restrict__ dh, const bf16 *__restrict__ h, int64_t n,
                            bf16 *__restrict__ dz, bf16 *__restrict__ dzt, float *__restrict__ db) {
    __shared__ bf16 tile[kTT][kTT + 2];
    __shared__ float colsum[8][kTT];
    const int64_t r0 = blockIdx.y * (int64_t)kTT;
    const int c0 = blockIdx.x * kTT, tx = threadIdx.x;
    float s0 = 0.f, s1 = 0.f;
    for (int j = threadIdx.y; j < kTT; j += blockDim.y) {
        const int64_t r = r0 + j;
        float2 v = make_float2(0.f, 0.f);
        if (r < n) {
            const int64_t o = r * kHid + c0 + 2 * tx;
            const float2 d = *reinterpret_cast<const float2 *>(dh + o);
            const __nv_bfloat162 hv = *reinterpret_cast<const __nv_bfloat162 *>(h + o);
            v.x = __bfloat162float(hv.x) > 0.f ? d.x : 0.f;
            v.y = __bfloat162float(hv.y) > 0.f ? d.y : 0.f;
            *reinterpret_cast<__nv_bfloat162 *>(dz + o) = __floats2bfloat162_rn(v.x, v.y);
        }
        tile[j][2 * tx] = __float2bfloat16(v.x);
        tile[j][2 * tx + 1] = __float2bfloat16(v.y);
        s0 += v.x;
        s1 += v.y;
    }
    colsum[threadIdx.y][2 * tx] = s0;
    colsum[threadIdx.y][2 * tx + 1] = s1;
    __syncthreads();
    const int64_t r = r0 + 2 * tx;
    for (int j = threadIdx.y; j < kTT; j += blockDim.y) {
        bf16 *d = dzt + (int64_t)(c0 + j) * n + r;
        if (r + 1 < n) {
            __nv_bfloat162 v;
            v.x = tile[2 * tx][j];
            v.y = tile[2 * tx + 1][j];
            if ((n & 1) == 0) *reinterpret_cast<__nv_bfloat162 *>(d) = v;  // 4-byte aligned
            else d[0] = v.x, d[1] = v.y;
        } else if (r < n) {
            d[0] = tile[2 * tx][j];
        }
    }
    if (threadIdx.y == 0) {
        for (int q = 0; q < 2; ++q) {
            float t = 0.f;
            for (int k = 0; k < 8; ++k) t += colsum[k][2 * tx + q];
            atomicAdd(db + c0 + 2 * tx + q, t);
        }
    }
}

// Where the BF16 copies of the four weight matrices go (W_l and W_l^T).
struct PackTargets {
    bf16 *wb[4], *wt[4];
};

// Adam (Kingma and Ba, 2015), bias-corrected, over the flat FP32 parameters;
// for an element of a weight matrix, its BF16 copies in W and W^T (what k_pack
// writes) in the same pass.
__global__ void k_adam_pack(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2, PackTargets pk) {
    const int64_t off[4] = {kOffW1, kOffW2, kOffW3, kOffW4};
    const int rows[4] = {kHid, kHid, kHid, kOut}, cols[4] = {kIn, kHid, kHid, kHid};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int64_t j = i - off[l];
            if (j >= 0 && j < (int64_t)rows[l] * cols[l]) {
                const bf16 b = __float2bfloat16(wi);
                pk.wb[l][j] = b;
                pk.wt[l][(j % cols[l]) * rows[l] + j / cols[l]] = b;
            }
        }
    }
}

// BF16 copies of a weight matrix [rows x cols] (FP32): W and W^T.
__global__ void k_pack(const float *__restrict__ w, int rows, int cols, bf16 *__restrict__ wb,
                       bf16 *__restrict__ wt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * cols) return;
    const int r = i / cols, c = i % cols;
    const bf16 b = __float2bfloat16(w[i]);
    wb[i] = b;
    if (wt) wt[(int64_t)c * rows + r] = b;
}

__global__ void k_take2(const float *__restrict__ y, int64_t n, float *__restrict__ out) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r < n) {
        out[2 * r] = y[r * kOut];
        out[2 * r + 1] = y[r * kOut + 1];
    }
}

// Rows idx[r] of x (BF16, kIn per row) and t (FP32, 2 per row) into rows r of
// xb and tb, r < n; an index outside 0..n_rows-1 gives a zero row.
__global__ void k_gather_rows(const uint4 *__restrict__ x, const float2 *__restrict__ t, int64_t n_rows,
                              const int32_t *__restrict__ idx, int64_t n, uint4 *__restrict__ xb,
                              float2 *__restrict__ tb) {
    constexpr int kChunks = kIn * 2 / 16;  // 16-byte chunks per input row
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n * kChunks;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = q / kChunks;
        const int c = (int)(q - r * kChunks);
        const int64_t src = idx[r];
        const bool in = src >= 0 && src < n_rows;
        xb[q] = in ? x[src * kChunks + c] : make_uint4(0, 0, 0, 0);
        if (c == 0) tb[r] = in ? t[src] : make_float2(0.f, 0.f);
    }
}

}  // namespace

struct llama_mlp {
    int device = 0;
    int64_t cap = 0;      // batch capacity (rows)
    int64_t steps = 0;    // Adam steps taken
    int64_t version = 0;  // bumped whenever the weights change (set_params, train_step)
    Buf w, g, m, v;       // FP32 parameters, gradients, Adam moments
    Buf wb[4], wt[4];     // BF16 W_l and W_l^T
    Buf h1, h2, h3, y;    // activations (BF16) and outputs (FP32, 64 per row)
    Buf h0t, h1t, h2t, h3t, dy, dyt, dh, dz, dzt;
    Buf part;             // FP32 partial products of the split-K weight gradients
    Buf xb, tb;           // one gathered mini-batch of inputs (BF16) and targets (FP32)
    int sms = 0;          // SMs of the device (sets the split of the weight gradients)
    std::string err;
};

namespace {

const int kRows[4] = {kHid, kHid, kHid, kOut}, kCols[4] = {kIn, kHid, kHid, kHid};
// the split-K partials of one weight gradient: up to 64 splits of a 256 x 256 product
constexpr size_t kPartBytes = 64 * sizeof(float) * kHid * kHid;

// dW = dz^T h (FP32 [rows x cols] into g), K = the batch: with so few output
// tiles the product is split over K (deterministic partial sums).
int weight_gradient(llama_mlp *m, const void *dzt, const void *ht, float *g, int rows, int cols, int64_t n,
                    cudaStream_t s) {
    int splits = splits_for(rows, cols, (int)n, m->sms);
    while (splits > 1 && (size_t)splits * rows * cols * sizeof(float) > kPartBytes) splits /= 2;
    return gemm_split_k(dzt, ht, g, rows, cols, (int)n, splits, m->part.as<float>(), kPartBytes, s);
}
const int64_t kOffW[4] = {kOffW1, kOffW2, kOffW3, kOffW4}, kOffB[4] = {kOffB1, kOffB2, kOffB3, kOffB4};

struct Guard {
    int prev = -1;
    explicit Guard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~Guard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

int fail(llama_mlp *m, int code, const char *what, cudaError_t e = cudaSuccess) {
    m->err = std::string(what) + (e != cudaSuccess ? std::string(": ") + cudaGetErrorString(e) : "");
    return code;
}

#define MLP_CUDA(m, call)                                                          \
    do {                                                                           \
        const cudaError_t e__ = (call);                                            \
        if (e__ != cudaSuccess)                                                    \
            return fail((m), e__ == cudaErrorMemoryAllocation ? LLAMA_ENOMEM : LLAMA_ECUDA, #call, e__); \
    } while (0)

#define MLP_RC(call)                 \
    do {                             \
        const int rc__ = (call);     \
        if (rc__ != LLAMA_OK) return rc__; \
    } while (0)

int pack_weights(llama_mlp *m, cudaStream_t s) {
    const float *w = m->w.as<float>();
    for (int l = 0; l < 4; ++l) {
        const int n = kRows[l] * kCols[l];
        k_pack<<<(n + 255) / 256, 256, 0, s>>>(w + kOffW[l], kRows[l], kCols[l], m->wb[l].as<bf16>(),
                                              m->wt[l].as<bf16>());
    }
    MLP_CUDA(m, cudaGetLastError());
    return LLAMA_OK;
}

void transpose(const bf16 *src, bf16 *dst, int64_t rows, int cols, cudaStream_t s) {
    const dim3 grid((unsigned)(cols / kTT), (unsigned)((rows + kTT - 1) / kTT));  // cols: 64 or 256
    k_transpose<<<grid, dim3(32, 8), 0, s>>>(src, dst, rows, cols);
}

// Forward pass over n rows of x (BF16 [n x 64]): h1, h2, h3 (BF16), y (FP32 [n x 64]).
int forward(llama_mlp *m, const void *x, int64_t n, cudaStream_t s) {
    const float *w = m->w.as<float>();
    MLP_RC(gemm(x, m->wb[0].p, w + kOffB1, m->h1.p, nullptr, n, kHid, kIn, LLAMA_GEMM_RELU, s));
    MLP_RC(gemm(m->h1.p, m->wb[1].p, w + kOffB2, m->h2.p, nullptr, n, kHid, kHid, LLAMA_GEMM_RELU, s));
    MLP_RC(gemm(m->h2.p, m->wb[2].p, w + kOffB3, m->h3.p, nullptr, n, kHid, kHid, LLAMA_GEMM_RELU, s));
    MLP_RC(gemm(m->h3.p, m->wb[3].p, w + kOffB4, nullptr, m->y.as<float>(), n, kOut, kHid, 0, s));
    return LLAMA_OK;
}

// Gradients of the mean loss into m->g (FP32, flat), after a forward pass.
int backward(llama_mlp *m, const void *x, const float *t, int64_t n, float w_fan, float *loss, cudaStream_t s) {
    float *g = m->g.as<float>();
    MLP_CUDA(m, cudaMemsetAsync(g, 0, sizeof(float) * kParams, s));
    k_loss_grad<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m->y.as<float>(), t, n, w_fan, m->dy.as<bf16>(),
                                                           g + kOffB4, loss);
    transpose(m->dy.as<bf16>(), m->dyt.as<bf16>(), n, kOut, s);
    transpose(static_cast<const bf16 *>(x), m->h0t.as<bf16>(), n, kIn, s);
    transpose(m->h1.as<bf16>(), m->h1t.as<bf16>(), n, kHid, s);
    transpose(m->h2.as<bf16>(), m->h2t.as<bf16>(), n, kHid, s);
    transpose(m->h3.as<bf16>(), m->h3t.as<bf16>(), n, kHid, s);
    MLP_CUDA(m, cudaGetLastError());
    // layer 4 (linear): dW4 = dy^T h3, dh3 = dy W4
    MLP_RC(weight_gradient(m, m->dyt.p, m->h3t.p, g + kOffW4, kOut, kHid, n, s));
    MLP_RC(gemm(m->dy.p, m->wt[3].p, nullptr, nullptr, m->dh.as<float>(), n, kHid, kOut, 0, s));
    const bf16 *hs[3] = {m->h1.as<bf16>(), m->h2.as<bf16>(), m->h3.as<bf16>()};
    const void *hts[4] = {m->h0t.p, m->h1t.p, m->h2t.p, m->h3t.p};
    const dim3 rgrid(kHid / kTT, (unsigned)((n + kTT - 1) / kTT));
    for (int l = 2; l >= 0; --l) {
        // through the ReLU of layer l+1, then dW = dz^T h_l and (below layer 1) dh_l = dz W
        k_relu_back<<<rgrid, dim3(32, 8), 0, s>>>(m->dh.as<float>(), hs[l], n, m->dz.as<bf16>(),
                                                 m->dzt.as<bf16>(), g + kOffB[l]);
        MLP_CUDA(m, cudaGetLastError());
        MLP_RC(weight_gradient(m, m->dzt.p, hts[l], g + kOffW[l], kHid, kCols[l], n, s));
        if (l > 0) MLP_RC(gemm(m->dz.p, m->wt[l].p, nullptr, nullptr, m->dh.as<float>(), n, kHid, kHid, 0, s));
    }
    return LLAMA_OK;
}

// One Adam step (bias-corrected) on m->g at learning rate lr, with the BF16
// copies of the weights written in the same pass.
int adam_step(llama_mlp *m, float lr, cudaStream_t s) {
    const int64_t step = ++m->steps;
    ++m->version;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - (float)std::pow((double)b1, (double)step), c2 = 1.f - (float)std::pow((double)b2, (double)step);
    PackTargets pk;
    for (int l = 0; l < 4; ++l) pk.wb[l] = m->wb[l].as<bf16>(), pk.wt[l] = m->wt[l].as<bf16>();
    k_adam_pack<<<592, 256, 0, s>>>(m->w.as<float>(), m->g.as<float>(), m->m.as<float>(), m->v.as<float>(),
                                    kParams, lr, b1, b2, 1e-8f, c1, c2, pk);
    MLP_CUDA(m, cudaGetLastError());
    return LLAMA_OK;
}

int check_batch(llama_mlp *m, const void *x, int64_t n, bool training) {
    if (!x) return fail(m, LLAMA_EINVAL, "null input");
    if (n < 1 || n > m->cap) return fail(m, LLAMA_EINVAL, "batch outside 1..max_batch");
    if (training && n % 128) return fail(m, LLAMA_EINVAL, "training batches must be a multiple of 128 rows");
    if (reinterpret_cast<uintptr_t>(x) & 15) return fail(m, LLAMA_EINVAL, "input not 16-byte aligned");
    return LLAMA_OK;
}

}  // namespace

extern "C" int llama_mlp_create(llama_mlp **out, int32_t device, int64_t max_batch) {
    if (!out) return LLAMA_EINVAL;
    *out = nullptr;
    if (max_batch < 128 || max_batch > (1 << 26)) return LLAMA_EINVAL;
    llama_mlp *m = new llama_mlp();
    m->device = device;
    m->cap = (max_batch + 127) / 128 * 128;
    Guard gd(device);
    const int64_t c = m->cap;
    cudaError_t e = cudaSuccess;
    auto A = [&](Buf &b, size_t bytes) { if (e == cudaSuccess) e = b.alloc(bytes); };
    A(m->w, 4 * kParams), A(m->g, 4 * kParams), A(m->m, 4 * kParams), A(m->v, 4 * kParams);
    for (int l = 0; l < 4; ++l) A(m->wb[l], 2 * kRows[l] * kCols[l]), A(m->wt[l], 2 * kRows[l] * kCols[l]);
    A(m->h1, 2 * c * kHid), A(m->h2, 2 * c * kHid), A(m->h3, 2 * c * kHid), A(m->y, 4 * c * kOut);
    A(m->h0t, 2 * c * kIn), A(m->h1t, 2 * c * kHid), A(m->h2t, 2 * c * kHid), A(m->h3t, 2 * c * kHid);
    A(m->dy, 2 * c * kOut), A(m->dyt, 2 * c * kOut), A(m->dh, 4 * c * kHid), A(m->dz, 2 * c * kHid);
    A(m->dzt, 2 * c * kHid);
    A(m->part, kPartBytes);
    A(m->xb, 2 * c * kIn), A(m->tb, 4 * c * 2);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&m->sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMemset(m->dy.p, 0, 2 * c * kOut);  // the loss writes columns 0 and 1 only
    if (e == cudaSuccess) e = cudaMemset(m->w.p, 0, 4 * kParams);
    if (e == cudaSuccess) e = cudaMemset(m->m.p, 0, 4 * kParams);
    if (e == cudaSuccess) e = cudaMemset(m->v.p, 0, 4 * kParams);
    if (e == cudaSuccess && pack_weights(m, nullptr) != LLAMA_OK) e = cudaErrorUnknown;
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete m;
        return e == cudaErrorMemoryAllocation ? LLAMA_ENOMEM : LLAMA_ECUDA;
    }
    *out = m;
    return LLAMA_OK;
}

extern "C" void llama_mlp_destroy(llama_mlp *m) {
    if (!m) return;
    Guard gd(m->device);
    delete m;
}

extern "C" int llama_mlp_set_params(llama_mlp *m, const float *params) {
    if (!m) return LLAMA_EINVAL;
    if (!params) return fail(m, LLAMA_EINVAL, "set_params: null params");
    Guard gd(m->device);
    MLP_CUDA(m, cudaMemcpy(m->w.p, params, 4 * kParams, cudaMemcpyHostToDevice));
    MLP_CUDA(m, cudaMemset(m->m.p, 0, 4 * kParams));
    MLP_CUDA(m, cudaMemset(m->v.p, 0, 4 * kParams));
    m->steps = 0;
    ++m->version;
    MLP_RC(pack_weights(m, nullptr));
    MLP_CUDA(m, cudaDeviceSynchronize());
    return LLAMA_OK;
}

extern "C" int llama_mlp_get_params(llama_mlp *m, float *params) {
    if (!m) return LLAMA_EINVAL;
    if (!params) return fail(m, LLAMA_EINVAL, "get_params: null params");
    Guard gd(m->device);
    MLP_CUDA(m, cudaDeviceSynchronize());
    MLP_CUDA(m, cudaMemcpy(params, m->w.p, 4 * kParams, cudaMemcpyDeviceToHost));
    return LLAMA_OK;
}

extern "C" int llama_mlp_forward(llama_mlp *m, const void *x, int64_t n, float *y, void *stream) {
    if (!m) return LLAMA_EINVAL;
    MLP_RC(check_batch(m, x, n, false));
    if (!y) return fail(m, LLAMA_EINVAL, "forward: null output");
    Guard gd(m->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MLP_RC(forward(m, x, n, s));
    k_take2<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m->y.as<float>(), n, y);
    MLP_CUDA(m, cudaGetLastError());
    return LLAMA_OK;
}

extern "C" int llama_mlp_gradients(llama_mlp *m, const void *x, const float *t, int64_t n, float w_fan,
                                   float *grads, float *loss, void *stream) {
    if (!m) return LLAMA_EINVAL;
    MLP_RC(check_batch(m, x, n, true));
    if (!t) return fail(m, LLAMA_EINVAL, "gradients: null targets");
    Guard gd(m->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (loss) MLP_CUDA(m, cudaMemsetAsync(loss, 0, sizeof(float), s));
    MLP_RC(forward(m, x, n, s));
    MLP_RC(backward(m, x, t, n, w_fan, loss, s));
    if (grads) MLP_CUDA(m, cudaMemcpyAsync(grads, m->g.p, 4 * kParams, cudaMemcpyDeviceToDevice, s));
    return LLAMA_OK;
}

extern "C" int llama_mlp_train_step(llama_mlp *m, const void *x, const float *t, int64_t n, float w_fan,
                                    float lr, float *loss, void *stream) {
    if (!m) return LLAMA_EINVAL;
    MLP_RC(check_batch(m, x, n, true));
    if (!t) return fail(m, LLAMA_EINVAL, "train_step: null targets");
    if (!(lr > 0.f) || lr > 1.f) return fail(m, LLAMA_EINVAL, "train_step: learning rate outside (0, 1]");
    Guard gd(m->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (loss) MLP_CUDA(m, cudaMemsetAsync(loss, 0, sizeof(float), s));
    MLP_RC(forward(m, x, n, s));
    MLP_RC(backward(m, x, t, n, w_fan, loss, s));
    return adam_step(m, lr, s);
}

extern "C" int llama_mlp_train_epoch(llama_mlp *m, const void *x, const float *t, int64_t n_rows,
                                     const int32_t *perm, int64_t n_batches, int64_t batch, float w_fan, float lr,
                                     float *loss_sum, void *stream) {
    if (!m) return LLAMA_EINVAL;
    if (!x || !t || !perm || n_rows < 1 || n_batches < 0) return fail(m, LLAMA_EINVAL, "train_epoch: bad arguments");
    if (batch < 128 || batch > m->cap || batch % 128) return fail(m, LLAMA_EINVAL, "train_epoch: bad batch size");
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(t)) & 15)
        return fail(m, LLAMA_EINVAL, "train_epoch: inputs not 16-byte aligned");
    if (!(lr > 0.f) || lr > 1.f) return fail(m, LLAMA_EINVAL, "train_epoch: learning rate outside (0, 1]");
    Guard gd(m->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t chunks = batch * (kIn * 2 / 16);
    const unsigned grid = (unsigned)std::min<int64_t>((chunks + 255) / 256, 4096);
    for (int64_t b = 0; b < n_batches; ++b) {
        k_gather_rows<<<grid, 256, 0, s>>>(static_cast<const uint4 *>(x), reinterpret_cast<const float2 *>(t), n_rows,
                                           perm + b * batch, batch, m->xb.as<uint4>(), m->tb.as<float2>());
        MLP_CUDA(m, cudaGetLastError());
        MLP_RC(forward(m, m->xb.p, batch, s));
        MLP_RC(backward(m, m->xb.p, m->tb.as<float>(), batch, w_fan, loss_sum, s));
        MLP_RC(adam_step(m, lr, s));
    }
    return LLAMA_OK;
}

extern "C" const char *llama_mlp_last_error(llama_mlp *m) { return m ? m->err.c_str() : "null network"; }

namespace sgk {
llama_mlp_view mlp_view(const llama_mlp *m) {
    llama_mlp_view v{};
    v.params = m->w.as<float>();
    for (int l = 0; l < 4; ++l) v.w16[l] = m->wb[l].p;
    v.device = m->device;
    v.version = m->version;
    return v;
}
}  // namespace sgk
