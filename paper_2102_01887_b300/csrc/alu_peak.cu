// alu_peak.cu -- measured ceiling of the scan's inner loop (the denominator
// of the scoring kernel's ALU roofline; no counterpart in the paper).
//
// The scan scores two configurations with one packed subtract of the latency
// ranks, one LOP3 that flags the infeasible half onto the objective ranks, and
// one per-half 16-bit minimum (cost-first), plus one PRMT in alpha mode.  This
// kernel issues exactly that instruction mix on operands held in registers
// (no loads), with enough independent chains per thread to hide latency, on
// every SM, so its rate is what the integer pipes sustain for the mix: the
// scan cannot score faster than this when every operand is already on chip.
// (One extra add per eight chain steps changes the subtrahend each iteration;
// the scan's own loads of rank vectors go to the load/store pipe.)
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/llama.h"

namespace {

constexpr int kChains = 8;  // independent running minima per thread
constexpr int kThreads = 256;

template <bool ALPHA>
__global__ void __launch_bounds__(kThreads) k_alu_peak(uint32_t *sink, int iters, uint32_t seed) {
    const uint32_t t = threadIdx.x + blockIdx.x * blockDim.x + seed;
    uint32_t best[kChains], lk[kChains], rk[kChains], dk[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
        best[j] = 0xFFFFFFFFu;
        lk[j] = 0x80008000u + ((t * 2654435761u + j) & 0x0FFF0FFFu);
        rk[j] = (t ^ (0x9E3779B9u * (j + 1))) & 0x7FFF7FFFu;
        dk[j] = rk[j] ^ 0x00FF00FFu;
    }
    // the per-invocation count changes every iteration (one add per kChains
    // chain steps), so the assembler cannot hoist the subtract or the LOP3
    uint32_t c2 = (t & 0x0FFFu) * 0x00010001u;
    for (int it = 0; it < iters; ++it) {
        asm volatile("add.u32 %0, %0, 0x00010001;" : "+r"(c2));
#pragma unroll
        for (int j = 0; j < kChains; ++j) {
            uint32_t d, k;
            asm volatile("sub.u32 %0, %1, %2;" : "=r"(d) : "r"(lk[j]), "r"(c2));
            if (ALPHA) {
                asm volatile("prmt.b32 %0, %1, 0, 0xBB99;" : "=r"(d) : "r"(d));
                asm volatile("lop3.b32 %0, %1, %2, %3, 0x6A;" : "=r"(k) : "r"(dk[j]), "r"(d), "r"(rk[j]));
            } else {
                asm volatile("lop3.b32 %0, %1, 0x80008000, %2, 0xEA;" : "=r"(k) : "r"(d), "r"(rk[j]));
            }
            asm volatile("min.u16x2 %0, %1, %2;" : "=r"(best[j]) : "r"(best[j]), "r"(k));
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) acc ^= best[j];
    if (acc == 0x12345678u) sink[0] = acc;  // keeps the chains live
}

}  // namespace

extern "C" int llama_alu_peak(int32_t device, int32_t mode, double *scores_per_s) {
    if (!scores_per_s || (mode != LLAMA_MODE_COST_FIRST && mode != LLAMA_MODE_ALPHA)) return LLAMA_EINVAL;
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return LLAMA_EINVAL;
    int sms = 0, per_sm = 0;
    const void *fn = mode == LLAMA_MODE_ALPHA ? (const void *)k_alu_peak<true> : (const void *)k_alu_peak<false>;
    uint32_t *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t s = nullptr;
    int rc = LLAMA_ECUDA;
    float best_ms = 1e30f;
    const int iters = 2048;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) goto done;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, 0) != cudaSuccess) goto done;
    if (cudaMalloc(&sink, 16) != cudaSuccess) goto done;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) goto done;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) goto done;
    {
        const int blocks = sms * std::max(1, per_sm);
        // kWarm back-to-back launches (tens of ms of full load) bring the SM
        // clock up from whatever the GPU was doing before; then the best of
        // kTimed single launches
        constexpr int kWarm = 40, kTimed = 20;
        for (int rep = 0; rep < kWarm + kTimed; ++rep) {
            if (rep >= kWarm) cudaEventRecord(e0, s);
            if (mode == LLAMA_MODE_ALPHA) k_alu_peak<true><<<blocks, kThreads, 0, s>>>(sink, iters, rep);
            else k_alu_peak<false><<<blocks, kThreads, 0, s>>>(sink, iters, rep);
            if (rep < kWarm) continue;
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) goto done;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            best_ms = std::min(best_ms, ms);
        }
        // two configurations per chain step
        *scores_per_s = 2.0 * kChains * (double)iters * blocks * kThreads / (best_ms * 1e-3);
        rc = cudaGetLastError() == cudaSuccess ? LLAMA_OK : LLAMA_ECUDA;
    }
done:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (sink) cudaFree(sink);
    if (prev >= 0) cudaSetDevice(prev);
    return rc;
}
