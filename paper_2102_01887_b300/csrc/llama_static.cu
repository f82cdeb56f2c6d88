// llama_static.cu -- llama_schedule_static: the scheduling call without any
// device allocation.
//
// Why it exists.  llama_schedule and llama_schedule_async keep their
// bucketing scratch in context-owned buffers that grow with cudaMalloc when
// a call needs more room.  Some callers cannot let a library allocate at call
// time: a serving loop whose device memory was carved up front by its own
// allocator (an extra cudaMalloc can fail or fragment it), a latency-bound
// loop that cannot absorb the implicit synchronisation of cudaMalloc/cudaFree,
// or code that runs where the CUDA allocator must not be entered at all.
// This entry point uses instead one fixed, file-scope device array: every GPU
// that loads the library holds it (about 4.2 MB) until the process exits.  The
// caller still passes inputs and outputs; the context's tables were copied to
// the device earlier by llama_set_profiles.
//
// Sharing.  Every call on a device uses the same array, and the array keeps
// the contents of the last call.  The counters and control words that must be
// zero when a call starts are zero: the array starts zeroed, the last kernel
// of every completed call clears them, and a call whose later launch fails
// clears them with memsets on its stream (enqueue_schedule) before returning
// ECUDA.  Calls that overlap on the GPU (two streams, or two contexts on one
// device, in flight at once) race on the array and give wrong results:
// serialise them.  The status of the last completed call (invalid
// invocations, a bounded wait that gave up) stays in the array's status
// words; llama_static_status reads it.
//
// Set-up.  The device address of the array is looked up once per device with
// cudaGetSymbolAddress, by the first call on that device, with that device
// current.  Make that first call before any stream capture.  The address is
// cached for the process: after cudaDeviceReset it would be stale, so the
// entry point must not be used again after a reset.
#include <mutex>
#include <string>

#include "llama_internal.cuh"

using namespace llama;

namespace {

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Layout of the array (offsets in bytes, each part 256-byte aligned).
constexpr size_t kMaxTiles = (size_t)LLAMA_STATIC_MAX_INV + (size_t)LLAMA_STATIC_MAX_OPS;
constexpr size_t kCntOff = 0;
constexpr size_t kCtrlOff = align256(kCntOff + 4 * (size_t)kCntStride * LLAMA_STATIC_MAX_OPS);
constexpr size_t kOpStartOff = align256(kCtrlOff + 8 * (size_t)(kCtrlWords + kStatusWords) + 16 * (size_t)kMaxBucketBlocks);
constexpr size_t kGopOff = align256(kOpStartOff + 4 * (size_t)(LLAMA_STATIC_MAX_OPS + 1));
constexpr size_t kSlotOff = align256(kGopOff + 4 * (size_t)LLAMA_STATIC_MAX_INV);
constexpr size_t kBEntOff = align256(kSlotOff + 4 * (size_t)LLAMA_STATIC_MAX_INV);
constexpr size_t kRbaseOff = align256(kBEntOff + 8 * (size_t)LLAMA_STATIC_MAX_INV);
constexpr size_t kTilesOff = align256(kRbaseOff + 8 * (size_t)LLAMA_STATIC_MAX_INV);
constexpr size_t kScratchBytes = align256(kTilesOff + 32 * kMaxTiles);

constexpr int kMaxDevices = 64;

}  // namespace

// In host code this name is only a host-side stand-in for the array; the
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

namespace {

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the array on `device`, which must be current.
cudaError_t scratch_address(int device, void **out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return cudaSuccess;
}

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

int cuda_error(llama_ctx *c, cudaError_t e, const char *what) {
    std::string msg = std::string("schedule_static: ") + what + ": " + cudaGetErrorString(e);
    return context_fail(c, LLAMA_ECUDA, msg.c_str());
}

}  // namespace

extern "C" int llama_schedule_static(llama_ctx *c, int64_t n_inv, const int32_t *dag,
                                     const int32_t *op_local, const int64_t *start_us,
                                     int64_t now_us, llama_decision *out, void *stream) {
    if (!c) return LLAMA_EINVAL;
    if (n_inv < 0 || n_inv > LLAMA_STATIC_MAX_INV)
        return context_fail(c, LLAMA_EINVAL,
                            "schedule_static: n_inv exceeds LLAMA_STATIC_MAX_INV (65536)");
    if (n_inv > 0 && (!dag || !op_local || !start_us || !out))
        return context_fail(c, LLAMA_EINVAL, "schedule_static: null invocation or output pointer");
    ContextView v;
    int rc = context_view(c, &v);
    if (rc) return rc;
    if (v.n_ops > LLAMA_STATIC_MAX_OPS)
        return context_fail(c, LLAMA_EINVAL,
                            "schedule_static: the profiles have more than LLAMA_STATIC_MAX_OPS (4096) operations");
    if (v.device < 0 || v.device >= kMaxDevices)
        return context_fail(c, LLAMA_EINVAL, "schedule_static: device ordinal above 63");
    if (n_inv == 0) return LLAMA_OK;

    CurrentDevice guard(v.device);
    unsigned char *base = nullptr;
    cudaError_t e = scratch_address(v.device, reinterpret_cast<void **>(&base));
    if (e != cudaSuccess) return cuda_error(c, e, "cudaGetSymbolAddress");
    BucketScratch S{};
    S.cnt = reinterpret_cast<int32_t *>(base + kCntOff);
    S.ctrl = reinterpret_cast<unsigned long long *>(base + kCtrlOff);
    S.status = S.ctrl + kCtrlWords;
    S.blk = reinterpret_cast<int4 *>(base + kCtrlOff + 8 * (size_t)(kCtrlWords + kStatusWords));
    S.op_start = reinterpret_cast<int32_t *>(base + kOpStartOff);
    S.gop = reinterpret_cast<int32_t *>(base + kGopOff);
    S.slot = reinterpret_cast<int32_t *>(base + kSlotOff);
    S.b_ent = reinterpret_cast<int2 *>(base + kBEntOff);
    S.rbase = reinterpret_cast<int64_t *>(base + kRbaseOff);
    S.tiles = reinterpret_cast<int4 *>(base + kTilesOff);

    // the counters and control words are zero: the array starts zeroed, and
    // every completed call, or a failed enqueue, leaves them cleared
    e = enqueue_schedule(v, S, n_inv, dag, op_local, start_us, now_us, out,
                         static_cast<cudaStream_t>(stream), nullptr);
    if (e != cudaSuccess) return cuda_error(c, e, "enqueue");
    context_set_launches(c, schedule_launches(v, S, n_inv));
    return LLAMA_OK;
}

extern "C" int llama_static_status(llama_ctx *c, void *stream, int64_t *invalid, int32_t *timeout) {
    if (!c) return LLAMA_EINVAL;
    ContextView v;
    const int rc = context_view(c, &v);
    if (rc) return rc;
    const int device = v.device;
    if (device < 0 || device >= kMaxDevices)
        return context_fail(c, LLAMA_EINVAL, "static_status: device ordinal above 63");
    CurrentDevice guard(device);
    unsigned char *base = nullptr;
    cudaError_t e = scratch_address(device, reinterpret_cast<void **>(&base));
    if (e != cudaSuccess) return cuda_error(c, e, "cudaGetSymbolAddress");
    unsigned long long st[kStatusWords] = {0, 0};
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    e = cudaMemcpyAsync(st, base + kCtrlOff + 8 * (size_t)kCtrlWords, sizeof(st), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(c, e, "status copy");
    if (invalid) *invalid = (int64_t)st[0];
    if (timeout) *timeout = st[1] ? 1 : 0;
    return LLAMA_OK;
}
