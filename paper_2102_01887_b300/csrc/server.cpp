// Serving loop: continuous batching of arriving invocations over several
// slots (stream + workspace + staging buffers each), so that batches formed
// while others run on the GPU overlap with them.  Host code only.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <mutex>
#include <vector>

#include "llama.h"
#include "llama_server.h"

namespace {

int64_t clock_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Pending {
    llama_request r;
    int64_t t_submit;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t begin = nullptr, end = nullptr;
    llama_ws *ws = nullptr;
    int32_t *h_dag = nullptr, *h_opl = nullptr, *d_dag = nullptr, *d_opl = nullptr;
    int64_t *h_start = nullptr, *d_start = nullptr;
    llama_decision *h_out = nullptr, *d_out = nullptr;
    // device addresses of the page-locked request arrays: the kernels read a
    // batch's requests in place (no copy launches); null if the host memory
    // is not mapped into the device's address space, then they are copied
    const int32_t *m_dag = nullptr, *m_opl = nullptr;
    const int64_t *m_start = nullptr;
    std::vector<int64_t> ids, t_submit;
    int64_t n = 0;
    bool busy = false;
};

}  // namespace

struct llama_server {
    llama_ctx *ctx = nullptr;
    int device = 0;
    llama_server_opts opts{};
    std::vector<Slot> slots;
    cudaEvent_t base = nullptr;
    std::mutex mu;
    std::deque<Pending> queue;
    std::deque<llama_result> ready;
    std::vector<std::pair<float, float>> intervals;  // device [begin, end] of every batch, ms after base
    llama_server_stats st{};
    bool failed = false;
};

namespace {

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

void free_slot(Slot &s) {
    if (s.ws) llama_ws_destroy(s.ws);
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.begin) cudaEventDestroy(s.begin);
    if (s.end) cudaEventDestroy(s.end);
    cudaFreeHost(s.h_dag);
    cudaFreeHost(s.h_opl);
    cudaFreeHost(s.h_start);
    cudaFreeHost(s.h_out);
    cudaFree(s.d_dag);
    cudaFree(s.d_opl);
    cudaFree(s.d_start);
    cudaFree(s.d_out);
    s = Slot{};
}

int init_slot(llama_server *srv, Slot &s, int64_t B) {
    if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&s.begin) != cudaSuccess || cudaEventCreate(&s.end) != cudaSuccess ||
        cudaMallocHost(&s.h_dag, 4 * B) != cudaSuccess || cudaMallocHost(&s.h_opl, 4 * B) != cudaSuccess ||
        cudaMallocHost(&s.h_start, 8 * B) != cudaSuccess ||
        cudaMallocHost(&s.h_out, sizeof(llama_decision) * B) != cudaSuccess ||
        cudaMalloc(&s.d_dag, 4 * B) != cudaSuccess || cudaMalloc(&s.d_opl, 4 * B) != cudaSuccess ||
        cudaMalloc(&s.d_start, 8 * B) != cudaSuccess ||
        cudaMalloc(&s.d_out, sizeof(llama_decision) * B) != cudaSuccess)
        return LLAMA_ENOMEM;
    void *md = nullptr, *mo = nullptr, *ms = nullptr;
    if (cudaHostGetDevicePointer(&md, s.h_dag, 0) == cudaSuccess &&
        cudaHostGetDevicePointer(&mo, s.h_opl, 0) == cudaSuccess &&
        cudaHostGetDevicePointer(&ms, s.h_start, 0) == cudaSuccess) {
        s.m_dag = static_cast<const int32_t *>(md);
        s.m_opl = static_cast<const int32_t *>(mo);
        s.m_start = static_cast<const int64_t *>(ms);
    } else {
        cudaGetLastError();
    }
    const int rc = llama_ws_create(srv->ctx, B, &s.ws);
    if (rc) return rc;
    s.ids.resize(B);
    s.t_submit.resize(B);
    return LLAMA_OK;
}

// Device bytes of one slot for batches of B requests (workspace and buffers).
int64_t slot_bytes(int64_t B) { return B * (4 + 4 + 8 + 24) + B * (4 + 4 + 4 + 4 * LLAMA_MAX_HW + 8 + 32) + (1 << 20); }

// Start a batch on free slot s with up to max_batch queued requests.
int launch(llama_server *srv, Slot &s) {
    int64_t n = 0, now_b = INT64_MIN;
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        n = std::min<int64_t>((int64_t)srv->queue.size(), srv->opts.max_batch);
        for (int64_t k = 0; k < n; ++k) {
            const Pending &q = srv->queue[k];
            s.ids[k] = q.r.id;
            s.t_submit[k] = q.t_submit;
            s.h_dag[k] = q.r.dag;
            s.h_opl[k] = q.r.op_local;
            s.h_start[k] = q.r.start_us;
            now_b = std::max(now_b, q.r.now_us);
        }
        // every request against its own now_us: shift its start by the batch's
        // now minus its own (elapsed time unchanged; an invalid start stays invalid)
        for (int64_t k = 0; k < n; ++k) s.h_start[k] += now_b - srv->queue[k].r.now_us;
        srv->queue.erase(srv->queue.begin(), srv->queue.begin() + n);
    }
    if (n == 0) return LLAMA_OK;
    s.n = n;
    cudaEventRecord(s.begin, s.stream);
    const bool mapped = s.m_dag && s.m_opl && s.m_start;
    if (!mapped && (cudaMemcpyAsync(s.d_dag, s.h_dag, 4 * n, cudaMemcpyHostToDevice, s.stream) != cudaSuccess ||
                    cudaMemcpyAsync(s.d_opl, s.h_opl, 4 * n, cudaMemcpyHostToDevice, s.stream) != cudaSuccess ||
                    cudaMemcpyAsync(s.d_start, s.h_start, 8 * n, cudaMemcpyHostToDevice, s.stream) != cudaSuccess))
        return LLAMA_ECUDA;
    // (the slot's host arrays are not rewritten before its end event: the slot is busy until then)
    const int rc = llama_schedule_ws_async(srv->ctx, s.ws, n, mapped ? s.m_dag : s.d_dag, mapped ? s.m_opl : s.d_opl,
                                           mapped ? s.m_start : s.d_start, now_b, s.d_out, s.stream);
    if (rc) return rc;
    if (cudaMemcpyAsync(s.h_out, s.d_out, sizeof(llama_decision) * n, cudaMemcpyDeviceToHost, s.stream) !=
        cudaSuccess)
        return LLAMA_ECUDA;
    cudaEventRecord(s.end, s.stream);
    s.busy = true;
    ++srv->st.batches;
    int in_flight = 0;
    for (const Slot &o : srv->slots) in_flight += o.busy;
    srv->st.max_in_flight = std::max(srv->st.max_in_flight, in_flight);
    return LLAMA_OK;
}

int collect(llama_server *srv, Slot &s) {
    const cudaError_t q = cudaEventQuery(s.end);
    if (q == cudaErrorNotReady) return LLAMA_OK;
    if (q != cudaSuccess) return LLAMA_ECUDA;
    const int64_t t = clock_ns();
    float b = 0.f, e = 0.f;
    if (cudaEventElapsedTime(&b, srv->base, s.begin) == cudaSuccess &&
        cudaEventElapsedTime(&e, srv->base, s.end) == cudaSuccess)
        srv->intervals.emplace_back(b, e);
    for (int64_t k = 0; k < s.n; ++k) {
        llama_result r;
        r.id = s.ids[k];
        r.decision = s.h_out[k];
        r.submit_ns = s.t_submit[k];
        r.done_ns = t;
        srv->ready.push_back(r);
    }
    srv->st.completed += s.n;
    s.busy = false;
    s.n = 0;
    return LLAMA_OK;
}

}  // namespace

extern "C" int llama_server_create(llama_ctx *ctx, const llama_server_opts *opts, llama_server **out) {
    if (!ctx || !opts || !out) return LLAMA_EINVAL;
    *out = nullptr;
    if (opts->max_batch < 1 || opts->max_batch > (1 << 20) || opts->slots < 0 || opts->slots > 64 ||
        opts->memory_budget < 0 || opts->max_queue < 0)
        return LLAMA_EINVAL;
    int device = 0;
    cudaGetDevice(&device);
    llama_server *srv = new llama_server();
    srv->ctx = ctx;
    srv->opts = *opts;
    if (!srv->opts.max_queue) srv->opts.max_queue = 1 << 24;
    int n_slots = opts->slots;
    if (n_slots == 0) {
        if (opts->memory_budget <= 0) {
            delete srv;
            return LLAMA_EINVAL;
        }
        n_slots = (int)std::min<int64_t>(64, opts->memory_budget / slot_bytes(opts->max_batch));
        if (n_slots < 1) {
            delete srv;
            return LLAMA_ENOMEM;
        }
    }
    srv->device = device;
    srv->slots.resize(n_slots);
    srv->st.slots = n_slots;
    int rc = cudaEventCreate(&srv->base) == cudaSuccess ? LLAMA_OK : LLAMA_ECUDA;
    for (int k = 0; rc == LLAMA_OK && k < n_slots; ++k) rc = init_slot(srv, srv->slots[k], opts->max_batch);
    if (rc == LLAMA_OK) {
        cudaEventRecord(srv->base, srv->slots[0].stream);
        if (cudaStreamSynchronize(srv->slots[0].stream) != cudaSuccess) rc = LLAMA_ECUDA;
    }
    if (rc != LLAMA_OK) {
        llama_server_destroy(srv);
        return rc;
    }
    *out = srv;
    return LLAMA_OK;
}

extern "C" void llama_server_destroy(llama_server *srv) {
    if (!srv) return;
    Guard g(srv->device);
    for (Slot &s : srv->slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        free_slot(s);
    }
    if (srv->base) cudaEventDestroy(srv->base);
    delete srv;
}

extern "C" int llama_server_submit(llama_server *srv, const llama_request *req, int64_t n) {
    if (!srv || n < 0 || (n > 0 && !req)) return LLAMA_EINVAL;
    const int64_t t = clock_ns();
    std::lock_guard<std::mutex> lock(srv->mu);
    if ((int64_t)srv->queue.size() + n > srv->opts.max_queue) {
        srv->st.refused += n;
        return LLAMA_EAGAIN;
    }
    for (int64_t k = 0; k < n; ++k) srv->queue.push_back(Pending{req[k], t});
    srv->st.submitted += n;
    srv->st.queue_peak = std::max<int64_t>(srv->st.queue_peak, (int64_t)srv->queue.size());
    return LLAMA_OK;
}

extern "C" int llama_server_poll(llama_server *srv, llama_result *out, int64_t max_out, int64_t *n_out) {
    if (!srv || !n_out || max_out < 0 || (max_out > 0 && !out)) return LLAMA_EINVAL;
    *n_out = 0;
    if (srv->failed) return LLAMA_ECUDA;
    Guard g(srv->device);
    for (Slot &s : srv->slots) {
        if (s.busy) {
            const int rc = collect(srv, s);
            if (rc) {
                srv->failed = true;
                return rc;
            }
        }
        if (!s.busy) {
            const int rc = launch(srv, s);
            if (rc) {
                srv->failed = true;
                return rc;
            }
        }
    }
    const int64_t k = std::min<int64_t>(max_out, (int64_t)srv->ready.size());
    for (int64_t i = 0; i < k; ++i) out[i] = srv->ready[i];
    srv->ready.erase(srv->ready.begin(), srv->ready.begin() + k);
    *n_out = k;
    return LLAMA_OK;
}

extern "C" int llama_server_drain(llama_server *srv, llama_result *out, int64_t max_out, int64_t *n_out,
                                  int64_t timeout_ms) {
    if (!srv || !n_out) return LLAMA_EINVAL;
    *n_out = 0;
    const int64_t deadline = clock_ns() + timeout_ms * 1000000;
    for (;;) {
        int64_t got = 0;
        const int rc = llama_server_poll(srv, out ? out + *n_out : nullptr, max_out - *n_out, &got);
        if (rc) return rc;
        *n_out += got;
        bool idle;
        {
            std::lock_guard<std::mutex> lock(srv->mu);
            idle = srv->queue.empty();
        }
        for (const Slot &s : srv->slots) idle = idle && !s.busy;
        if (idle && (srv->ready.empty() || *n_out == max_out)) return LLAMA_OK;
        if (clock_ns() > deadline) return LLAMA_ETIMEOUT;
    }
}

extern "C" int llama_server_stats_get(llama_server *srv, llama_server_stats *st) {
    if (!srv || !st) return LLAMA_EINVAL;
    *st = srv->st;
    // device-time overlap of the batches seen so far
    std::vector<std::pair<float, float>> iv = srv->intervals;
    std::sort(iv.begin(), iv.end());
    int64_t overlapped = 0;
    double busy = 0.0, cur_b = -1.0, cur_e = -1.0, max_end = -1e30;
    for (size_t k = 0; k < iv.size(); ++k) {
        const bool ov = iv[k].first < max_end || (k + 1 < iv.size() && iv[k + 1].first < iv[k].second);
        overlapped += ov;
        max_end = std::max<double>(max_end, iv[k].second);
        if (iv[k].first > cur_e) {
            if (cur_e > cur_b) busy += cur_e - cur_b;
            cur_b = iv[k].first;
            cur_e = iv[k].second;
        } else {
            cur_e = std::max<double>(cur_e, iv[k].second);
        }
    }
    if (cur_e > cur_b) busy += cur_e - cur_b;
    st->overlapped = overlapped;
    st->device_busy_ms = busy;
    st->device_span_ms = iv.empty() ? 0.0 : max_end - iv.front().first;
    return LLAMA_OK;
}
