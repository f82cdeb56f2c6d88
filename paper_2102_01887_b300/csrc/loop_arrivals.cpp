// loop_arrivals.cpp -- native arrival processes for serving (no counterpart in
// the paper), on the calling host thread, timed by the steady clock:
//  * the device-resident loop: requests submitted to its ring as their arrival
//    times come, its records polled (the driver thread runs the ticks);
//  * the learned surrogate's path: continuous batching, each call taking every
//    request that arrived while the previous one ran.
// Host code only (the surrogate's calls enqueue its kernels).
#include <cuda_runtime.h>

#include <chrono>
#include <cstdint>
#include <vector>

#include "../../include/llama_loop.h"
#include "../../include/llama_server.h"
#include "../../include/llama_surrogate.h"

extern "C" int llama_loop_run_arrivals(llama_loop *loop, const llama_loop_request *req, const int64_t *arrive_ns,
                                       int64_t n, int64_t id0, int64_t timeout_ns, int64_t *spec_ns,
                                       int64_t *commit_ns) {
    if (!loop || n < 0 || (n > 0 && (!req || !arrive_ns || !spec_ns || !commit_ns)) || timeout_ns < 1)
        return LLAMA_EINVAL;
    for (int64_t k = 0; k < n; ++k) {
        if (req[k].id != id0 + k) return LLAMA_EINVAL;  // records are matched to requests by id
        if (k > 0 && arrive_ns[k] < arrive_ns[k - 1]) return LLAMA_EINVAL;
        spec_ns[k] = commit_ns[k] = -1;
    }
    constexpr int64_t kBatch = 4096;  // requests per submit, records per poll at most
    std::vector<llama_loop_result> res(kBatch);
    const auto t0 = std::chrono::steady_clock::now();
    const auto since = [&] {
        return (int64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0)
            .count();
    };
    int64_t submitted = 0, seen = 0;
    while (seen < 2 * n) {
        const int64_t t = since();
        // every request whose time has come, as far as the ring has room (a full
        // ring never blocks: the rest waits for the next pass)
        while (submitted < n && arrive_ns[submitted] <= t) {
            int64_t m = 1;
            while (m < kBatch && submitted + m < n && arrive_ns[submitted + m] <= t) ++m;
            const int rc = llama_loop_submit(loop, req + submitted, m);
            if (rc == LLAMA_EAGAIN) break;
            if (rc != LLAMA_OK) return rc;
            submitted += m;
        }
        int64_t got = 0;
        const int rc = llama_loop_poll(loop, res.data(), kBatch, &got);
        if (rc != LLAMA_OK) return rc;
        if (got > 0) {
            const int64_t now = since();
            for (int64_t r = 0; r < got; ++r) {
                const int64_t k = res[r].id - id0;
                if (k < 0 || k >= n) continue;
                if (res[r].kind == LLAMA_LOOP_SPECULATED && spec_ns[k] < 0) spec_ns[k] = now, ++seen;
                else if (res[r].kind == LLAMA_LOOP_COMMITTED && commit_ns[k] < 0) commit_ns[k] = now, ++seen;
                else if (res[r].kind == LLAMA_LOOP_REJECTED && spec_ns[k] < 0) spec_ns[k] = commit_ns[k] = now, seen += 2;
            }
        }
        if (since() > timeout_ns) break;  // records not seen by then stay -1
    }
    return LLAMA_OK;
}

extern "C" int llama_sg_run_arrivals(llama_sg *sg, const void *cfg_x, const void *inv_x, const int32_t *dag,
                                     const int32_t *op_local, const int64_t *start_us, int64_t n,
                                     const int64_t *arrive_ns, int64_t now_us, int64_t max_batch,
                                     llama_decision *out, llama_decision *host_out, void *stream, int64_t *done_ns) {
    if (!sg || n < 0 || max_batch < 1) return LLAMA_EINVAL;
    if (n > 0 && (!cfg_x || !inv_x || !dag || !op_local || !start_us || !arrive_ns || !out || !host_out || !done_ns))
        return LLAMA_EINVAL;
    for (int64_t k = 1; k < n; ++k)
        if (arrive_ns[k] < arrive_ns[k - 1]) return LLAMA_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const auto t0 = std::chrono::steady_clock::now();
    const auto since = [&] {
        return (int64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0)
            .count();
    };
    constexpr int64_t kRow = 64 * 2;  // bytes of one BF16 feature row
    int64_t k = 0;
    while (k < n) {
        const int64_t t = since();
        int64_t j = k;
        while (j < n && j - k < max_batch && arrive_ns[j] <= t) ++j;
        if (j == k) continue;  // nothing has arrived yet
        const int64_t m = j - k;
        int rc = llama_sg_schedule(sg, cfg_x, static_cast<const char *>(inv_x) + k * kRow, m, dag + k,
                                   op_local + k, start_us + k, now_us + t / 1000, out, stream);
        if (rc != LLAMA_OK) return rc;
        if (cudaMemcpyAsync(host_out, out, sizeof(llama_decision) * m, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return LLAMA_ECUDA;
        const int64_t now = since();
        for (int64_t q = k; q < j; ++q) done_ns[q] = now;
        k = j;
    }
    return LLAMA_OK;
}
