// count_rate.cu -- measured floor of the bucketing step's per-op counting (no
// counterpart in the paper; reported beside the bucketing kernel's roofline).
//
// The bucketing kernel counts every invocation for its operation with one
// returning atomic add on a per-op counter (one counter per 128-byte line),
// four invocations per thread in flight.  This kernel runs that pattern alone:
// n operation indices spread over n_counters counters, loaded coalesced, four
// returning atomics in flight per thread, every rank stored -- and, for the
// floor of its memory part, the same loads and stores without the atomics.
// The bucketing kernel cannot count faster than the first.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/llama.h"

namespace {

constexpr int kThreads = 256;
constexpr int kInFlight = 4;         // atomics per thread per round
constexpr int kCounterStride = 32;   // int32 slots between counters: one 128-byte line each

// Operation index of element i: a multiplicative hash of i (with a
// xorshift-multiply finaliser), reduced mod n_counters.
__global__ void k_fill_ops(int32_t *g, int64_t n, int32_t n_counters) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t x = (uint32_t)i * 2654435761u + 0x9E3779B9u;
        x ^= x >> 15;
        x *= 0x2C1B3C6Du;
        x ^= x >> 12;
        g[i] = (int32_t)(x % (uint32_t)n_counters);
    }
}

template <bool ATOMIC>
__global__ void __launch_bounds__(kThreads) k_count_rate(const int32_t *g, int64_t n, int32_t *cnt, int32_t *slot) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < n; i0 += kInFlight * stride) {
        int32_t gg[kInFlight], s[kInFlight];
#pragma unroll
        for (int j = 0; j < kInFlight; ++j) gg[j] = i0 + j * stride < n ? g[i0 + j * stride] : -1;
#pragma unroll
        for (int j = 0; j < kInFlight; ++j)
            s[j] = gg[j] < 0 ? 0 : ATOMIC ? atomicAdd(&cnt[(int64_t)gg[j] * kCounterStride], 1) : gg[j] + 1;
#pragma unroll
        for (int j = 0; j < kInFlight; ++j)
            if (gg[j] >= 0) slot[i0 + j * stride] = s[j];
    }
}

}  // namespace

extern "C" int llama_count_rate(int32_t device, int64_t n, int32_t n_counters, double *atomic_us,
                                double *stream_us) {
    if (!atomic_us || !stream_us || n < 1 || n > LLAMA_MAX_INV || n_counters < 1) return LLAMA_EINVAL;
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return LLAMA_EINVAL;
    int sms = 0, per_sm = 0;
    int32_t *g = nullptr, *cnt = nullptr, *slot = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t s = nullptr;
    int rc = LLAMA_ECUDA;
    const size_t cnt_bytes = sizeof(int32_t) * kCounterStride * (size_t)n_counters;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) goto done;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count_rate<true>, kThreads, 0) != cudaSuccess)
        goto done;
    if (cudaMalloc(&g, sizeof(int32_t) * (size_t)n) != cudaSuccess ||
        cudaMalloc(&slot, sizeof(int32_t) * (size_t)n) != cudaSuccess || cudaMalloc(&cnt, cnt_bytes) != cudaSuccess)
        goto done;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) goto done;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) goto done;
    {
        // as many blocks as the bucketing kernel runs: four per SM, at most
        const int blocks = sms * std::min(4, std::max(1, per_sm));
        k_fill_ops<<<blocks, kThreads, 0, s>>>(g, n, n_counters);
        float best[2] = {1e30f, 1e30f};
        for (int rep = 0; rep < 24; ++rep) {
            const bool atomic = rep & 1;
            cudaMemsetAsync(cnt, 0, cnt_bytes, s);  // outside the timed region
            cudaEventRecord(e0, s);
            if (atomic) k_count_rate<true><<<blocks, kThreads, 0, s>>>(g, n, cnt, slot);
            else k_count_rate<false><<<blocks, kThreads, 0, s>>>(g, n, cnt, slot);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) goto done;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep >= 4) best[atomic] = std::min(best[atomic], ms);  // the first launches warm up
        }
        *atomic_us = 1e3 * best[1];
        *stream_us = 1e3 * best[0];
        rc = cudaGetLastError() == cudaSuccess ? LLAMA_OK : LLAMA_ECUDA;
    }
done:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (g) cudaFree(g);
    if (cnt) cudaFree(cnt);
    if (slot) cudaFree(slot);
    if (prev >= 0) cudaSetDevice(prev);
    return rc;
}
