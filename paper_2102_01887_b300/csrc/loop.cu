// loop.cu -- C ABI of the device-resident serving loop (include/llama_loop.h):
// early speculation and late commit (Section 4.3) with priority-based commit
// (Section 4.4).  The host only writes requests into a page-locked ring,
// launches ticks (k_loop_tick, kernels.cu) and reads result records from a
// second page-locked ring; every queue, sum and slot lives on the device.
#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <chrono>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "llama_internal.cuh"

using namespace llama;

namespace {

struct CurrentDevice {
    int prev = -1;
    explicit CurrentDevice(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~CurrentDevice() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

bool pow2(int64_t x) { return x >= 2 && (x & (x - 1)) == 0; }

}  // namespace

struct llama_loop {
    llama_ctx *ctx = nullptr;
    int device = 0;
    int32_t n_hw = 0;
    llama_loop_opts opts{};
    cudaStream_t stream = nullptr;
    // device memory
    std::vector<void *> dev_bufs;
    // page-locked, mapped host memory
    llama_loop_request *h_ring = nullptr;
    llama_loop_result *h_res = nullptr;
    LoopCtl *h_ctl = nullptr;
    std::atomic<int64_t> tail{0};  // requests written into the ring (published after the entries)
    int64_t res_read = 0;          // records taken by poll
    // the driver thread (llama_loop_start): ticks launched back to back
    std::thread driver;
    std::atomic<bool> running{false};
    std::atomic<int> driver_error{0};
    int64_t launched = 0;          // ticks enqueued (driver or llama_loop_tick)
    std::vector<int32_t> res_total;
    LoopDev L{};
    DevProblem P{};

    template <class T>
    cudaError_t dalloc(T **p, size_t count) {
        void *q = nullptr;
        const cudaError_t e = cudaMalloc(&q, sizeof(T) * (count ? count : 1));
        if (e == cudaSuccess) dev_bufs.push_back(q);
        *p = static_cast<T *>(q);
        return e;
    }
    void release() {
        running.store(false);
        if (driver.joinable()) driver.join();
        if (stream) cudaStreamSynchronize(stream);
        for (void *p : dev_bufs) cudaFree(p);
        dev_bufs.clear();
        if (h_ring) cudaFreeHost(h_ring);
        if (h_res) cudaFreeHost(h_res);
        if (h_ctl) cudaFreeHost(h_ctl);
        h_ring = nullptr;
        h_res = nullptr;
        h_ctl = nullptr;
        if (stream) cudaStreamDestroy(stream);
        stream = nullptr;
    }
};

namespace {

int loop_fail(llama_loop *lp, int code, const std::string &msg) {
    return context_fail(lp->ctx, code, ("loop: " + msg).c_str());
}

int loop_cuda(llama_loop *lp, cudaError_t e, const char *what) {
    return loop_fail(lp, e == cudaErrorMemoryAllocation ? LLAMA_ENOMEM : LLAMA_ECUDA,
                     std::string(what) + ": " + cudaGetErrorString(e));
}

// The context's current tables (staircase included), Eq. 3's minima tables and
// the critical paths computed on the loop's stream, and the problem view the
// ticks use (P.q = the loop's queueing-time array).
int loop_tables(llama_loop *lp) {
    int rc = context_ensure_stair(lp->ctx);
    if (rc) return rc;
    ContextView v;
    if ((rc = context_view(lp->ctx, &v))) return rc;
    cudaError_t e = cudaSuccess;
    if (!lp->L.objmin) {  // sized by the profiles, which a loop keeps
        int64_t *om = nullptr;
        if ((e = lp->dalloc(&om, (size_t)v.n_hw * (size_t)(v.P.n_cfg + v.n_ops))) != cudaSuccess)
            return loop_cuda(lp, e, "Eq. 3 minima tables");
        lp->L.objmin = om;
    }
    e = enqueue_encode_objmin(v, lp->L.objmin, lp->stream);
    if (e == cudaSuccess) e = enqueue_critical_paths(v, lp->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lp->stream);
    if (e != cudaSuccess) return loop_cuda(lp, e, "Eq. 3 minima tables and critical paths");
    lp->P = v.P;
    lp->P.q = lp->L.q;
    return LLAMA_OK;
}

}  // namespace

extern "C" int llama_loop_create(llama_ctx *ctx, const llama_loop_opts *opts, llama_loop **out) {
    if (!ctx || !opts || !out) return LLAMA_EINVAL;
    *out = nullptr;
    ContextView v;
    int rc = context_view(ctx, &v);
    if (rc) return rc;
    const int H = v.n_hw;
    if (!v.P.batch || !v.P.res || !v.P.res_total)
        return context_fail(ctx, LLAMA_EINVAL, "loop: the profiles carry no batch sizes or resources "
                                               "(batch, res, res_total: Eq. 1's penalty, Eq. 2, Eq. 3)");
    if (opts->slots < 1 || opts->slots > (1 << 22) || !pow2(opts->ring) || opts->ring > (1 << 24) ||
        !pow2(opts->results) || opts->results > (1 << 24) || opts->max_admit < 1 ||
        opts->max_admit > LLAMA_LOOP_MAX_ADMIT)
        return context_fail(ctx, LLAMA_EINVAL, "loop: slots, ring, results or max_admit out of range");
    int32_t cq_sum = 0, cq_max = 1;
    for (int h = 0; h < H; ++h) {
        if (opts->cq_cap[h] < 1) return context_fail(ctx, LLAMA_EINVAL, "loop: every cq_cap must be at least 1");
        cq_sum += opts->cq_cap[h];
        cq_max = std::max(cq_max, opts->cq_cap[h]);
    }
    if (cq_sum > LLAMA_LOOP_MAX_COMMIT)
        return context_fail(ctx, LLAMA_EINVAL, "loop: commit-queue capacities sum above LLAMA_LOOP_MAX_COMMIT");

    llama_loop *lp = new (std::nothrow) llama_loop();
    if (!lp) return LLAMA_ENOMEM;
    lp->ctx = ctx;
    lp->device = v.device;
    lp->n_hw = H;
    lp->opts = *opts;
    CurrentDevice guard(v.device);
    auto fail = [&](int code) {
        lp->release();
        delete lp;
        return code;
    };
    cudaError_t e = cudaStreamCreateWithFlags(&lp->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail(loop_cuda(lp, e, "stream"));
    LoopDev &L = lp->L;
    const int32_t S = opts->slots;
    if ((e = lp->dalloc(&L.st, 1)) != cudaSuccess || (e = lp->dalloc(&L.free_stack, S)) != cudaSuccess ||
        (e = lp->dalloc(&L.slot_id, S)) != cudaSuccess || (e = lp->dalloc(&L.slot_start, S)) != cudaSuccess ||
        (e = lp->dalloc(&L.slot_dag, S)) != cudaSuccess || (e = lp->dalloc(&L.slot_opl, S)) != cudaSuccess ||
        (e = lp->dalloc(&L.slot_lr_spec, S)) != cudaSuccess ||
        (e = lp->dalloc(&L.slot_lr_commit, S)) != cudaSuccess ||
        (e = lp->dalloc(&L.sq, (size_t)H * S)) != cudaSuccess ||
        (e = lp->dalloc(&L.cq, (size_t)H * cq_max)) != cudaSuccess ||
        (e = lp->dalloc(&L.q, LLAMA_MAX_HW)) != cudaSuccess)
        return fail(loop_cuda(lp, e, "device state"));
    if ((e = cudaHostAlloc(&lp->h_ring, sizeof(llama_loop_request) * opts->ring, cudaHostAllocMapped)) != cudaSuccess ||
        (e = cudaHostAlloc(&lp->h_res, sizeof(llama_loop_result) * opts->results, cudaHostAllocMapped)) !=
            cudaSuccess ||
        (e = cudaHostAlloc(&lp->h_ctl, sizeof(LoopCtl), cudaHostAllocMapped)) != cudaSuccess)
        return fail(loop_cuda(lp, e, "page-locked rings"));
    std::memset(lp->h_ctl, 0, sizeof(LoopCtl));
    void *dp = nullptr;
    if ((e = cudaHostGetDevicePointer(&dp, lp->h_ring, 0)) != cudaSuccess) return fail(loop_cuda(lp, e, "ring"));
    L.ring = static_cast<const llama_loop_request *>(dp);
    if ((e = cudaHostGetDevicePointer(&dp, lp->h_res, 0)) != cudaSuccess) return fail(loop_cuda(lp, e, "results"));
    L.res = static_cast<llama_loop_result *>(dp);
    if ((e = cudaHostGetDevicePointer(&dp, lp->h_ctl, 0)) != cudaSuccess) return fail(loop_cuda(lp, e, "control"));
    L.ctl = static_cast<LoopCtl *>(dp);
    L.ring_mask = opts->ring - 1;
    L.res_cap = opts->results;
    L.slots = S;
    L.cq_stride = cq_max;
    L.max_admit = opts->max_admit;
    for (int h = 0; h < LLAMA_MAX_HW; ++h) L.cq_cap[h] = h < H ? opts->cq_cap[h] : 1;
    // initial state: empty queues, every slot free (slot 0 taken first)
    LoopState st{};
    st.free_top = S;
    std::vector<int32_t> stack(S);
    for (int32_t i = 0; i < S; ++i) stack[i] = S - 1 - i;
    lp->res_total.assign(H, 1);
    if ((e = cudaMemcpy(L.st, &st, sizeof(st), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(L.free_stack, stack.data(), 4 * (size_t)S, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(L.q, 0, 8 * LLAMA_MAX_HW)) != cudaSuccess ||
        (e = cudaMemcpy(lp->res_total.data(), v.P.res_total, 4 * (size_t)H, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return fail(loop_cuda(lp, e, "initial state"));
    if ((rc = loop_tables(lp))) return fail(rc);
    *out = lp;
    return LLAMA_OK;
}

extern "C" void llama_loop_destroy(llama_loop *lp) {
    if (!lp) return;
    CurrentDevice guard(lp->device);
    lp->release();
    delete lp;
}

extern "C" int llama_loop_submit(llama_loop *lp, const llama_loop_request *req, int64_t n) {
    if (!lp || n < 0 || (n > 0 && !req)) return LLAMA_EINVAL;
    const int64_t taken = (int64_t)*reinterpret_cast<volatile unsigned long long *>(&lp->h_ctl->head);
    const int64_t tail = lp->tail.load(std::memory_order_relaxed);
    if (tail - taken + n > lp->opts.ring) return -6;  // LLAMA_EAGAIN: the ring lacks room
    const int64_t mask = lp->opts.ring - 1;
    for (int64_t k = 0; k < n; ++k) lp->h_ring[(tail + k) & mask] = req[k];
    // the entries before the tail that publishes them (and before any tick that reads them)
    lp->tail.store(tail + n, std::memory_order_seq_cst);
    return LLAMA_OK;
}

extern "C" int llama_loop_tick(llama_loop *lp, int64_t now_us, const int32_t *dispatch) {
    if (!lp) return LLAMA_EINVAL;
    if (lp->running.load()) return loop_fail(lp, LLAMA_EINVAL, "tick: the driver thread is running");
    LoopTickArgs a{};
    a.now = now_us;
    a.limit = lp->tail.load(std::memory_order_seq_cst);
    for (int h = 0; h < lp->n_hw; ++h) {
        a.dispatch[h] = dispatch ? dispatch[h] : 0;
        if (a.dispatch[h] < 0) return loop_fail(lp, LLAMA_EINVAL, "tick: negative dispatch count");
    }
    CurrentDevice guard(lp->device);
    nvtxRangePushA("llama:loop_tick");
    std::atomic_thread_fence(std::memory_order_seq_cst);
    const cudaError_t e = enqueue_loop_tick(lp->P, lp->L, a, lp->stream);
    nvtxRangePop();
    if (e != cudaSuccess) return loop_cuda(lp, e, "tick launch");
    ++lp->launched;
    return LLAMA_OK;
}

namespace {

// One pause of a waiting loop (the core's spin-wait hint where there is one).
inline void cpu_relax() {
#if defined(__x86_64__) || defined(__i386__)
    __builtin_ia32_pause();
#else
    std::this_thread::yield();
#endif
}

// The driver thread: a tick whenever fewer than in_flight are queued, at the
// steady clock's time (now_us at the start, then the microseconds elapsed);
// every tick applies the same dispatch counts.  It spins (a pause per poll of
// the mapped control words) while ticks are queued, since a sleep of a few
// microseconds lasts tens on a general-purpose kernel and would let the queue
// run dry; with nothing pending on the device and nothing new in the ring it
// keeps spinning for a while, then sleeps between polls.
void drive(llama_loop *lp, int64_t now0, int in_flight, LoopTickArgs a) {
    cudaSetDevice(lp->device);
    const auto t0 = std::chrono::steady_clock::now();
    volatile LoopCtl *ctl = lp->h_ctl;
    constexpr int kIdleSpins = 1 << 16;  // polls before an idle loop starts to sleep
    int idle_spins = 0;
    while (lp->running.load(std::memory_order_relaxed)) {
        const int64_t done = (int64_t)ctl->ticks;
        const int64_t limit = lp->tail.load(std::memory_order_seq_cst);
        const bool idle = done == lp->launched && (int64_t)ctl->head == limit && ctl->inflight == 0;
        if (lp->launched - done >= in_flight || idle) {
            if (idle && ++idle_spins > kIdleSpins) std::this_thread::sleep_for(std::chrono::microseconds(20));
            else cpu_relax();
            continue;
        }
        idle_spins = 0;
        a.now = now0 + std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0).count();
        a.limit = limit;
        nvtxRangePushA("llama:loop_tick");
        const cudaError_t e = enqueue_loop_tick(lp->P, lp->L, a, lp->stream);
        nvtxRangePop();
        if (e != cudaSuccess) {
            lp->driver_error.store((int)e);
            lp->running.store(false);
            break;
        }
        ++lp->launched;
    }
}

}  // namespace

extern "C" int llama_loop_start(llama_loop *lp, int64_t now_us, int32_t ticks_in_flight, const int32_t *dispatch) {
    if (!lp) return LLAMA_EINVAL;
    if (lp->running.load()) return loop_fail(lp, LLAMA_EINVAL, "start: the driver thread is running");
    if (ticks_in_flight < 1 || ticks_in_flight > 64)
        return loop_fail(lp, LLAMA_EINVAL, "start: ticks_in_flight outside 1..64");
    LoopTickArgs a{};
    for (int h = 0; h < lp->n_hw; ++h) {
        a.dispatch[h] = dispatch ? dispatch[h] : 0;
        if (a.dispatch[h] < 0) return loop_fail(lp, LLAMA_EINVAL, "start: negative dispatch count");
    }
    lp->driver_error.store(0);
    lp->running.store(true);
    lp->driver = std::thread(drive, lp, now_us, (int)ticks_in_flight, a);
    return LLAMA_OK;
}

extern "C" int llama_loop_stop(llama_loop *lp) {
    if (!lp) return LLAMA_EINVAL;
    lp->running.store(false);
    if (lp->driver.joinable()) lp->driver.join();
    CurrentDevice guard(lp->device);
    const cudaError_t e = cudaStreamSynchronize(lp->stream);
    if (e != cudaSuccess) return loop_cuda(lp, e, "stop");
    const int de = lp->driver_error.load();
    if (de) return loop_cuda(lp, (cudaError_t)de, "driver tick launch");
    return LLAMA_OK;
}

extern "C" int llama_loop_poll(llama_loop *lp, llama_loop_result *out, int64_t max_out, int64_t *n_out) {
    if (!lp || !n_out || max_out < 0 || (max_out > 0 && !out)) return LLAMA_EINVAL;
    const int64_t count = (int64_t)*reinterpret_cast<volatile unsigned long long *>(&lp->h_ctl->res_count);
    std::atomic_thread_fence(std::memory_order_acquire);  // the records the count publishes
    const int64_t n = std::min<int64_t>(count - lp->res_read, max_out);
    const int64_t mask = lp->opts.results - 1;
    for (int64_t k = 0; k < n; ++k) out[k] = lp->h_res[(lp->res_read + k) & mask];
    lp->res_read += n;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    *reinterpret_cast<volatile unsigned long long *>(&lp->h_ctl->res_read) = (unsigned long long)lp->res_read;
    *n_out = n;
    return LLAMA_OK;
}

extern "C" int64_t llama_loop_ticks_done(llama_loop *lp) {
    if (!lp) return -1;
    return (int64_t)*reinterpret_cast<volatile unsigned long long *>(&lp->h_ctl->ticks);
}

extern "C" int llama_loop_sync(llama_loop *lp) {
    if (!lp) return LLAMA_EINVAL;
    CurrentDevice guard(lp->device);
    const cudaError_t e = cudaStreamSynchronize(lp->stream);
    return e == cudaSuccess ? LLAMA_OK : loop_cuda(lp, e, "sync");
}

extern "C" int llama_loop_state_get(llama_loop *lp, llama_loop_state *out) {
    if (!lp || !out) return LLAMA_EINVAL;
    CurrentDevice guard(lp->device);
    LoopState st{};
    cudaError_t e = cudaStreamSynchronize(lp->stream);
    if (e == cudaSuccess) e = cudaMemcpy(&st, lp->L.st, sizeof(st), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return loop_cuda(lp, e, "state");
    std::memset(out, 0, sizeof(*out));
    out->ticks = st.ticks;
    out->submitted = lp->tail.load();
    out->admitted = st.admitted;
    out->rejected = st.rejected;
    out->committed = st.committed;
    out->dispatched = st.dispatched;
    out->results = st.res_count;
    out->results_dropped = st.dropped;
    out->free_slots = st.free_top;
    for (int h = 0; h < lp->n_hw; ++h) {
        out->sq_len[h] = (int32_t)(st.sq_tail[h] - st.sq_head[h]);
        out->cq_len[h] = (int32_t)(st.cq_tail[h] - st.cq_head[h]);
        const unsigned __int128 s = st.s_sq[h] + st.s_cq[h];
        const unsigned __int128 cap = (unsigned __int128)INT32_MAX * (uint32_t)lp->res_total[h];
        out->q_us[h] = s >= cap ? INT32_MAX : (int64_t)((uint64_t)s / (uint32_t)lp->res_total[h]);
    }
    return LLAMA_OK;
}

extern "C" int llama_loop_refresh(llama_loop *lp) {
    if (!lp) return LLAMA_EINVAL;
    CurrentDevice guard(lp->device);
    const cudaError_t e = cudaStreamSynchronize(lp->stream);
    if (e != cudaSuccess) return loop_cuda(lp, e, "refresh");
    return loop_tables(lp);
}
