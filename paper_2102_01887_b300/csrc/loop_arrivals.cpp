// loop_arrivals.cpp -- a native arrival process for the serving loop (no
// counterpart in the paper): requests are submitted to the loop's ring as their
// arrival times come and the records are polled, on the calling host thread,
// each request's speculative and commit records timed by the steady clock.
// The driver thread (llama_loop_start) must be running.  Host code only.
#include <chrono>
#include <cstdint>
#include <thread>
#include <vector>

#include "../../include/llama_loop.h"
#include "../../include/llama_server.h"

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
