// Scheduling with the learned latency surrogate in place of the profile table.
//
// For every pending invocation i and every configuration x of its operation,
// the network predicts the log latency factor r(i, x) from the configuration's
// features and the invocation's content features; the predicted latency and
// cost are the profiled ones times e^r, and the decision is the cost-first
// selection of Eq. 1 over those predictions, each against slack(i, lambda(x))
// (Algorithm 1, through the critical path of the profiled reference
// latencies).  The first layer splits by linearity: z1(i, x) = A[x] + B[i] with
// A = (configuration features) W1^T and B = (content features) W1^T + b1, the
// other input columns being zero in each; so a pair costs one ReLU of a sum
// and two 256 x 256 products (tensor cores; a persistent kernel keeps each
// layer's weights in shared memory), the last layer and the selection running
// in the epilogue of the second product.
#include <cub/cub.cuh>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "llama_internal.cuh"
#include "llama_surrogate.h"
#include "sg_internal.cuh"

using namespace sgk;

namespace {

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t n) {
        if (n <= bytes) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
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

// Backend of every configuration (its segment).
__global__ void k_cfg_backend(llama::DevProblem P, int8_t *lam) {
    const int v = blockIdx.x, H = P.n_hw;
    const int64_t c0 = P.cfg_off[v];
    const int n = (int)(P.cfg_off[v + 1] - c0);
    const int32_t *hw = P.hw_off + (int64_t)v * (H + 1);
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
        int h = 0;
        while (h + 1 < H && x >= hw[h + 1]) ++h;
        lam[c0 + x] = (int8_t)h;
    }
}

// Grouping of the invocations by operation: the key of invocation i is its
// operation (n_ops when it has no decision, so it sorts last), the value i; the
// number of its pairs is kept and added to the total.
__global__ void k_pair_keys(llama::DevProblem P, int64_t n_inv, const int32_t *dag, const int32_t *op_local,
                            const int32_t *slack, int32_t *key, int32_t *idx, int64_t *npairs,
                            unsigned long long *total) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    unsigned k = 0;
    if (i == n_inv) npairs[i] = 0;  // the exclusive scan's last value is the total
    if (i < n_inv) {
        int32_t g = P.n_ops;
        if (slack[i * P.n_hw] >= 0) {
            g = P.dag_op_off[dag[i]] + op_local[i];
            k = (unsigned)(P.cfg_off[g + 1] - P.cfg_off[g]);
        }
        key[i] = g;
        idx[i] = (int32_t)i;
        npairs[i] = k;
    }
    const unsigned w = __reduce_add_sync(0xffffffffu, k);
    if ((threadIdx.x & 31) == 0 && w) atomicAdd(total, (unsigned long long)w);
}

// Rows of every invocation in operation order: its pairs rounded up to whole
// 128-row tiles (entry n_inv is 0: the exclusive scan's last value is the total).
__global__ void k_pair_rows(llama::DevProblem P, int64_t n_inv, const int32_t *key, int64_t *nrows) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k > n_inv) return;
    int64_t r = 0;
    if (k < n_inv && key[k] < P.n_ops) {
        const int32_t g = key[k];
        r = (P.cfg_off[g + 1] - P.cfg_off[g] + kTileRows - 1) / kTileRows * kTileRows;
    }
    nrows[k] = r;
}

// The rows of the k-th invocation in operation order (one block each): each
// pair's selection record (invocation, op-local index, profiled latency, slack
// on the configuration's backend; invocation -1 on a padding row) and profiled
// cost, every tile's first configuration row and invocation, and the
// invocation's first row.
__global__ void k_pair_index(llama::DevProblem P, const int32_t *key, const int32_t *idx, const int64_t *row_off,
                             const int32_t *slack, const int8_t *__restrict__ lam, int64_t *inv_row,
                             int4 *__restrict__ pair_sel, int64_t *__restrict__ pair_cost, int2 *__restrict__ tile_info) {
    const int64_t k = blockIdx.x;
    const int32_t i = idx[k], g = key[k];
    if (g >= P.n_ops) {
        if (threadIdx.x == 0) inv_row[i] = -1;
        return;
    }
    const int64_t c0 = P.cfg_off[g], r0 = row_off[k];
    const int n = (int)(P.cfg_off[g + 1] - c0), nr = (int)(row_off[k + 1] - r0);
    if (threadIdx.x == 0) inv_row[i] = r0;
    for (int x = threadIdx.x; x < nr; x += blockDim.x) {
        if (x < n) {
            const int64_t gc = c0 + x;
            pair_sel[r0 + x] = make_int4(i, x, P.lat[gc], slack[(int64_t)i * P.n_hw + lam[gc]]);
            pair_cost[r0 + x] = P.cost[gc];
        } else {
            pair_sel[r0 + x] = make_int4(-1, 0, 0, 0);
        }
        if (x % kTileRows == 0) tile_info[(r0 + x) / kTileRows] = make_int2((int)(c0 + x), i);
    }
}

// Predictions of the last call in invocation order (pairs of invocation i at
// pair_off[i] ..), from the rows in operation order.
__global__ void k_pair_compact(int64_t n_inv, const int64_t *pair_off, const int64_t *inv_row,
                               const int32_t *lhat_rows, const int64_t *chat_rows, int32_t *lhat, int64_t *chat) {
    const int64_t i = blockIdx.x;
    const int64_t p0 = pair_off[i], n = pair_off[i + 1] - p0, r0 = inv_row[i];
    for (int64_t x = threadIdx.x; x < n; x += blockDim.x) {
        if (lhat) lhat[p0 + x] = lhat_rows[r0 + x];
        if (chat) chat[p0 + x] = chat_rows[r0 + x];
    }
}

// The decision of every invocation from its best key.
__global__ void k_sg_decode(llama::DevProblem P, int64_t n_inv, const int32_t *dag, const int32_t *op_local,
                            const int32_t *slack, const int64_t *inv_row, const unsigned long long *best,
                            const int32_t *lhat, const int64_t *chat, const int8_t *lam, llama_decision *out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_inv) return;
    llama_decision d;
    if (slack[i * P.n_hw] < 0) {
        d.cfg = -1;
        d.lat = 0;
        d.cost = 0;
        d.slack = 0;
        d.flags = LLAMA_FLAG_INVALID;
    } else {
        const int32_t g = P.dag_op_off[dag[i]] + op_local[i];
        const int32_t x = (int32_t)(best[i] & 0x1FFFull);
        const int64_t p = inv_row[i] + x;
        d.cfg = x;
        d.lat = lhat[p];
        d.cost = chat[p];
        d.slack = slack[i * P.n_hw + lam[P.cfg_off[g] + x]];
        d.flags = d.lat < d.slack ? LLAMA_FLAG_FEASIBLE : 0;
    }
    out[i] = d;
}

}  // namespace

struct llama_sg {
    llama_ctx *ctx = nullptr;
    llama_mlp *net = nullptr;
    int device = 0;
    int64_t max_inv = 0, max_pairs = 0;
    // A: configuration part of layer 1 (BF16), B: invocation part (FP32); rows of
    // the pair layers in operation order, 128 per tile
    Buf A, B, h2, pair_sel, pair_cost, lhat, chat, tile_info, key, key_sorted, idx, idx_sorted, npairs, nrows,
        row_off, inv_row, pair_off, best, slack, lam, scan_tmp, total;
    int64_t last_pairs = 0, last_n_inv = 0;
    float margin = 0.f;
    // layer 1's configuration part A (and each configuration's backend) depends
    // only on the configuration features, the profiles and the weights: it is
    // kept across calls while these are the same
    const void *a_src = nullptr;
    const int64_t *a_cfg_off = nullptr;
    const int32_t *a_hw_off = nullptr;
    int64_t a_ncfg = -1, a_version = -1;
    std::string err;
    size_t cap_rows = 0;  // pair rows the pair buffers hold
};

namespace {

int sg_fail(llama_sg *s, int code, const std::string &what, cudaError_t e = cudaSuccess) {
    s->err = what + (e != cudaSuccess ? std::string(": ") + cudaGetErrorString(e) : "");
    return code;
}

#define SG_CUDA(s, call)                                                                              \
    do {                                                                                              \
        const cudaError_t e__ = (call);                                                               \
        if (e__ != cudaSuccess)                                                                       \
            return sg_fail((s), e__ == cudaErrorMemoryAllocation ? LLAMA_ENOMEM : LLAMA_ECUDA, #call, e__); \
    } while (0)

#define SG_RC(s, call, what)                          \
    do {                                              \
        const int rc__ = (call);                      \
        if (rc__ != LLAMA_OK) return sg_fail((s), rc__, what); \
    } while (0)

}  // namespace

namespace {

constexpr size_t kReserveInv = 4096;  // invocations whose row padding is reserved at creation

// Pair buffers for `rows` pair rows (h2, selection records and costs,
// predictions, tile descriptors).
cudaError_t reserve_rows(llama_sg *s, size_t rows) {
    rows = std::max<size_t>(rows, kTileRows);
    cudaError_t e = cudaSuccess;
    const auto A = [&](Buf &b, size_t n) {
        if (e == cudaSuccess) e = b.ensure(n);
    };
    A(s->h2, 2 * rows * kHid), A(s->pair_sel, 16 * rows), A(s->pair_cost, 8 * rows), A(s->lhat, 4 * rows);
    A(s->chat, 8 * rows), A(s->tile_info, 8 * (rows / kTileRows + 1));
    if (e == cudaSuccess) s->cap_rows = rows;
    return e;
}

}  // namespace

extern "C" int llama_sg_create(llama_sg **out, llama_ctx *ctx, llama_mlp *net, int64_t max_inv, int64_t max_pairs) {
    if (!out) return LLAMA_EINVAL;
    *out = nullptr;
    if (!ctx || !net || max_inv < 1 || max_inv > (1 << 24) || max_pairs < 128 || max_pairs > (1ll << 30))
        return LLAMA_EINVAL;
    llama_sg *s = new llama_sg();
    s->ctx = ctx;
    s->net = net;
    s->device = mlp_view(net).device;
    s->max_inv = max_inv;
    s->max_pairs = max_pairs;
    // the scratch of every call, allocated here so that a call normally
    // allocates nothing (an allocation inside a call synchronises the device
    // and stalls every request queued behind it): the per-invocation arrays and
    // the sort and scan scratch for max_inv invocations, and pair rows (whole
    // tiles per invocation) for max_pairs pairs and the padding of up to
    // kReserveInv invocations -- a call that needs more rows grows them
    // geometrically (reserve_rows)
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != s->device) cudaSetDevice(s->device);
    const size_t ni = (size_t)max_inv;
    cudaError_t e = reserve_rows(s, (size_t)max_pairs + (size_t)(kTileRows - 1) * std::min<size_t>(ni, kReserveInv));
    const auto A = [&](Buf &b, size_t n) {
        if (e == cudaSuccess) e = b.ensure(n);
    };
    A(s->B, 4 * ni * kHid), A(s->slack, 4 * ni * LLAMA_MAX_HW), A(s->key, 4 * ni), A(s->key_sorted, 4 * ni);
    A(s->idx, 4 * ni), A(s->idx_sorted, 4 * ni), A(s->npairs, 8 * (ni + 1)), A(s->nrows, 8 * (ni + 1));
    A(s->row_off, 8 * (ni + 1)), A(s->inv_row, 8 * ni), A(s->best, 8 * ni), A(s->total, 8);
    size_t t_sort = 0, t_scan = 0;  // for max_inv items and keys of up to 32 bits
    if (e == cudaSuccess)
        e = cub::DeviceRadixSort::SortPairs(nullptr, t_sort, s->key.as<int32_t>(), s->key_sorted.as<int32_t>(),
                                            s->idx.as<int32_t>(), s->idx_sorted.as<int32_t>(), (int)max_inv, 0, 32);
    if (e == cudaSuccess)
        e = cub::DeviceScan::ExclusiveSum(nullptr, t_scan, s->nrows.as<int64_t>(), s->row_off.as<int64_t>(),
                                          (int)(max_inv + 1));
    A(s->scan_tmp, std::max(t_sort, t_scan));
    if (prev >= 0 && prev != s->device) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return e == cudaErrorMemoryAllocation ? LLAMA_ENOMEM : LLAMA_ECUDA;
    }
    *out = s;
    return LLAMA_OK;
}

extern "C" void llama_sg_destroy(llama_sg *s) { delete s; }

extern "C" int llama_sg_schedule(llama_sg *s, const void *cfg_x, const void *inv_x, int64_t n_inv,
                                 const int32_t *dag, const int32_t *op_local, const int64_t *start_us,
                                 int64_t now_us, llama_decision *out, void *stream) {
    if (!s) return LLAMA_EINVAL;
    if (n_inv < 0 || n_inv > s->max_inv) return sg_fail(s, LLAMA_EINVAL, "schedule: n_inv outside 0..max_inv");
    if (n_inv == 0) {
        s->last_pairs = s->last_n_inv = 0;
        return LLAMA_OK;
    }
    if (!cfg_x || !inv_x || !dag || !op_local || !start_us || !out)
        return sg_fail(s, LLAMA_EINVAL, "schedule: null pointer");
    llama::ContextView v;
    SG_RC(s, llama::context_view(s->ctx, &v), "schedule: the scheduling context is not ready");
    const llama_mlp_view nv = mlp_view(s->net);
    if (nv.device != v.device) return sg_fail(s, LLAMA_EINVAL, "schedule: network and context on different GPUs");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != v.device) cudaSetDevice(v.device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int H = v.n_hw;
    const int64_t n_cfg = v.P.n_cfg;  // the context's configuration count (host)
    const size_t ni = (size_t)s->max_inv;
    SG_CUDA(s, s->A.ensure(2 * (size_t)n_cfg * kHid));
    SG_CUDA(s, s->lam.ensure((size_t)n_cfg));
    SG_CUDA(s, s->B.ensure(4 * ni * kHid));
    SG_CUDA(s, s->slack.ensure(4 * ni * H));
    SG_CUDA(s, s->key.ensure(4 * ni));
    SG_CUDA(s, s->key_sorted.ensure(4 * ni));
    SG_CUDA(s, s->idx.ensure(4 * ni));
    SG_CUDA(s, s->idx_sorted.ensure(4 * ni));
    SG_CUDA(s, s->npairs.ensure(8 * (ni + 1)));
    SG_CUDA(s, s->nrows.ensure(8 * (ni + 1)));
    SG_CUDA(s, s->row_off.ensure(8 * (ni + 1)));
    SG_CUDA(s, s->inv_row.ensure(8 * ni));
    SG_CUDA(s, s->best.ensure(8 * ni));
    SG_CUDA(s, s->total.ensure(8));
    // a1 + a2 on the profiled reference latencies
    llama::k_critical_paths<<<std::max(1, (v.n_dags + 7) / 8), 256, 0, st>>>(v.P, v.topo, v.lvl_off, v.dag_lvl);
    llama::k_slack<<<(unsigned)std::min<int64_t>((n_inv + 255) / 256, 65535), 256, 0, st>>>(
        v.P, n_inv, dag, op_local, start_us, now_us, s->slack.as<int32_t>());
    const bool a_cached = s->a_src == cfg_x && s->a_ncfg == n_cfg && s->a_version == nv.version &&
                          s->a_cfg_off == v.P.cfg_off && s->a_hw_off == v.P.hw_off;
    if (!a_cached) k_cfg_backend<<<v.n_ops, 256, 0, st>>>(v.P, s->lam.as<int8_t>());
    SG_CUDA(s, cudaMemsetAsync(s->total.p, 0, 8, st));
    k_pair_keys<<<(unsigned)((n_inv + 256) / 256), 256, 0, st>>>(v.P, n_inv, dag, op_local, s->slack.as<int32_t>(),
                                                                 s->key.as<int32_t>(), s->idx.as<int32_t>(),
                                                                 s->npairs.as<int64_t>(),
                                                                 s->total.as<unsigned long long>());
    SG_CUDA(s, cudaGetLastError());
    // invocations grouped by operation, so that the tiles running at one time
    // read the same configuration rows
    int bits = 1;
    while ((1ll << bits) <= (int64_t)v.n_ops) ++bits;
    size_t t_sort = 0, t_scan = 0;
    SG_CUDA(s, cub::DeviceRadixSort::SortPairs(nullptr, t_sort, s->key.as<int32_t>(), s->key_sorted.as<int32_t>(),
                                               s->idx.as<int32_t>(), s->idx_sorted.as<int32_t>(), (int)n_inv, 0,
                                               bits, st));
    SG_CUDA(s, cub::DeviceScan::ExclusiveSum(nullptr, t_scan, s->nrows.as<int64_t>(), s->row_off.as<int64_t>(),
                                             (int)(n_inv + 1), st));
    SG_CUDA(s, s->scan_tmp.ensure(std::max(t_sort, t_scan)));
    SG_CUDA(s, cub::DeviceRadixSort::SortPairs(s->scan_tmp.p, t_sort, s->key.as<int32_t>(),
                                               s->key_sorted.as<int32_t>(), s->idx.as<int32_t>(),
                                               s->idx_sorted.as<int32_t>(), (int)n_inv, 0, bits, st));
    k_pair_rows<<<(unsigned)((n_inv + 256) / 256), 256, 0, st>>>(v.P, n_inv, s->key_sorted.as<int32_t>(),
                                                                 s->nrows.as<int64_t>());
    SG_CUDA(s, cudaGetLastError());
    SG_CUDA(s, cub::DeviceScan::ExclusiveSum(s->scan_tmp.p, t_scan, s->nrows.as<int64_t>(), s->row_off.as<int64_t>(),
                                             (int)(n_inv + 1), st));
    int64_t pairs = 0, rows = 0;
    SG_CUDA(s, cudaMemcpyAsync(&pairs, s->total.p, 8, cudaMemcpyDeviceToHost, st));
    SG_CUDA(s, cudaMemcpyAsync(&rows, s->row_off.as<int64_t>() + n_inv, 8, cudaMemcpyDeviceToHost, st));
    SG_CUDA(s, cudaStreamSynchronize(st));
    if (pairs > s->max_pairs) return sg_fail(s, LLAMA_EINVAL, "schedule: more (invocation, configuration) pairs than max_pairs");
    s->last_pairs = pairs;
    s->last_n_inv = n_inv;
    if ((size_t)rows > s->cap_rows) SG_CUDA(s, reserve_rows(s, std::max<size_t>((size_t)rows, 2 * s->cap_rows)));
    // first layer, split: A = configurations . W1^T (BF16), B = contents . W1^T + b1
    if (!a_cached) {
        SG_RC(s, gemm(cfg_x, nv.w16[0], nullptr, s->A.p, nullptr, n_cfg, kHid, kIn, 0, st), "layer 1 (configurations)");
        s->a_src = cfg_x;
        s->a_ncfg = n_cfg;
        s->a_version = nv.version;
        s->a_cfg_off = v.P.cfg_off;
        s->a_hw_off = v.P.hw_off;
    }
    SG_RC(s, gemm(inv_x, nv.w16[0], nv.params + kOffB1, nullptr, s->B.as<float>(), n_inv, kHid, kIn, 0, st),
          "layer 1 (contents)");
    SG_CUDA(s, cudaMemsetAsync(s->best.p, 0xFF, 8 * (size_t)n_inv, st));
    k_pair_index<<<(unsigned)n_inv, 256, 0, st>>>(v.P, s->key_sorted.as<int32_t>(), s->idx_sorted.as<int32_t>(),
                                                  s->row_off.as<int64_t>(), s->slack.as<int32_t>(),
                                                  s->lam.as<int8_t>(), s->inv_row.as<int64_t>(),
                                                  s->pair_sel.as<int4>(), s->pair_cost.as<int64_t>(),
                                                  s->tile_info.as<int2>());
    SG_CUDA(s, cudaGetLastError());
    if (rows > 0) {
        SG_RC(s, mlp_layer_first(s->A.p, n_cfg, s->B.as<float>(), s->tile_info.as<int2>(), nv.w16[1],
                                 nv.params + kOffB2, s->h2.p, rows, st),
              "layers 1 and 2");
        SelectArgs a;
        a.w4 = nv.params + kOffW4;
        a.b4 = nv.params + kOffB4;
        a.pair_sel = s->pair_sel.as<int4>();
        a.pair_cost = s->pair_cost.as<int64_t>();
        a.margin = s->margin;
        a.best = s->best.as<unsigned long long>();
        a.lhat = s->lhat.as<int32_t>();
        a.chat = s->chat.as<int64_t>();
        SG_RC(s, mlp_layer_select(s->h2.p, nv.w16[2], nv.params + kOffB3, rows, a, st), "layer 3 and selection");
    }
    k_sg_decode<<<(unsigned)((n_inv + 255) / 256), 256, 0, st>>>(
        v.P, n_inv, dag, op_local, s->slack.as<int32_t>(), s->inv_row.as<int64_t>(),
        s->best.as<unsigned long long>(), s->lhat.as<int32_t>(), s->chat.as<int64_t>(), s->lam.as<int8_t>(), out);
    SG_CUDA(s, cudaGetLastError());
    if (prev >= 0 && prev != v.device) cudaSetDevice(prev);
    return LLAMA_OK;
}

extern "C" int64_t llama_sg_last_pairs(llama_sg *s) { return s ? s->last_pairs : -1; }

extern "C" int llama_sg_invalidate(llama_sg *s) {
    if (!s) return LLAMA_EINVAL;
    s->a_src = nullptr;
    s->a_ncfg = -1;
    return LLAMA_OK;
}

extern "C" int llama_sg_set_margin(llama_sg *s, float margin) {
    if (!s) return LLAMA_EINVAL;
    if (!(margin >= 0.f && margin <= 1.f)) return sg_fail(s, LLAMA_EINVAL, "set_margin: margin outside [0, 1]");
    s->margin = margin;
    return LLAMA_OK;
}

extern "C" int llama_sg_predictions(llama_sg *s, int32_t *lhat, int64_t *chat, int64_t *pair_off, int64_t n_inv,
                                    void *stream) {
    if (!s) return LLAMA_EINVAL;
    if (n_inv != s->last_n_inv) return sg_fail(s, LLAMA_EINVAL, "predictions: n_inv is not the last call's");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n_inv == 0) {
        if (pair_off) SG_CUDA(s, cudaMemsetAsync(pair_off, 0, 8, st));
        return LLAMA_OK;
    }
    // pair offsets in invocation order, then the rows gathered into them
    SG_CUDA(s, s->pair_off.ensure(8 * (size_t)(s->max_inv + 1)));
    size_t tmp = 0;
    SG_CUDA(s, cub::DeviceScan::ExclusiveSum(nullptr, tmp, s->npairs.as<int64_t>(), s->pair_off.as<int64_t>(),
                                             (int)(n_inv + 1), st));
    SG_CUDA(s, s->scan_tmp.ensure(tmp));
    SG_CUDA(s, cub::DeviceScan::ExclusiveSum(s->scan_tmp.p, tmp, s->npairs.as<int64_t>(), s->pair_off.as<int64_t>(),
                                             (int)(n_inv + 1), st));
    if ((lhat || chat) && s->last_pairs > 0) {
        k_pair_compact<<<(unsigned)n_inv, 256, 0, st>>>(n_inv, s->pair_off.as<int64_t>(), s->inv_row.as<int64_t>(),
                                                        s->lhat.as<int32_t>(), s->chat.as<int64_t>(), lhat, chat);
        SG_CUDA(s, cudaGetLastError());
    }
    if (pair_off)
        SG_CUDA(s, cudaMemcpyAsync(pair_off, s->pair_off.p, 8 * (size_t)(n_inv + 1), cudaMemcpyDeviceToDevice, st));
    return LLAMA_OK;
}

extern "C" const char *llama_sg_last_error(llama_sg *s) { return s ? s->err.c_str() : "null surrogate"; }
