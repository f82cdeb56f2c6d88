// llama_host.cu -- C ABI of the scheduling step (include/llama.h): argument
// validation, DAG levelling, padded table layout, device memory, launches.
#include <cub/cub.cuh>

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "llama_internal.cuh"

using namespace llama;

namespace {

// Owning device buffer.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    cudaError_t alloc(size_t n) {
        release();
        if (n == 0) n = 16;
        cudaError_t e = cudaMalloc(&p, n);
        if (e == cudaSuccess) bytes = n; else p = nullptr;
        return e;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// Makes the context's device current for the duration of an API call.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// An NVTX range over an API call (shown by Nsight tools; costs nothing when no
// tool is attached).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

}  // namespace

// Scratch of one scheduling call at a time: per-op counters and bucket
// starts, per-invocation bucket entries, the tile list and the control and
// status words.  Counters and control words are zero between calls.
struct Workspace {
    DevBuf cnt, ctrl, op_start, gop, slot, b_ent, rbase, tiles, b_cnt;
    int64_t cap_inv = 0, cap_tiles = 0;
    int32_t cap_ops = 0;
};

struct llama_ctx {
    llama_opts opts{};
    int num_sms = 0;
    int max_smem_optin = 0;
    int64_t l2_bytes = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t order_ev = nullptr;  // orders the context's own stream after table updates on other streams
    std::string err = "no error";

    // DAGs
    bool dags_set = false;
    int32_t n_dags = 0, n_ops_dag = 0;
    DevBuf dag_op_off, row_ptr, col, slo, dag_info, topo, lvl_off, dag_lvl;
    // host copies of the DAG structure (for the packed per-DAG layout)
    std::vector<int32_t> h_dag_op_off, h_row_ptr, h_col, h_topo, h_lvl_off, h_dag_lvl;
    std::vector<int64_t> h_ref_gidx;
    DevBuf dag_pack, dag_pack_off, ord_info, ord_cbase, dec, dfast;
    // staircase method (built on demand, see llama_set_method)
    int32_t method = LLAMA_METHOD_SCAN;
    bool stair_ready = false;
    DevBuf stair, stair_off;
    std::vector<int32_t> h_dn;     // distinct latencies per op (as set; feedback changes them on the device)
    std::vector<int32_t> h_npad;   // padded table entries per op
    std::vector<int32_t> h_ncfg;   // configurations per op
    int32_t max_n = 0, sort_cap = 1;
    size_t sort_smem = 0, lat_smem = 0;
    DevBuf ord_pos;                // bucket-order position of every op
    // feedback scratch
    DevBuf fb_keys, fb_idx, fb_keys2, fb_idx2, fb_touched, fb_rejected, fb_tmp;
    // commit-order scratch
    DevBuf co_aff, co_aff2, co_lam, co_lam2, co_idx, co_idx2, co_tmp;

    // profiles
    bool prof_set = false;
    int32_t n_ops = 0, max_npad = 0;
    int64_t n_cfg = 0, n_pad = 0;
    DevBuf cfg_off, hw_off, lat, cost, ref_cfg, batch, res, res_total;
    DevBuf pad_off, seg_pad, lrb, dlat, dlat_n, dpiv, dpiv2, rf, df, inv, fast, op_order, ref_gidx;
    int64_t mean_npad = 0;
    DevBuf ref, cp, cp_magic;
    DevBuf q_dev;  // [LLAMA_MAX_HW] queueing time per backend, read by the kernels
    DevBuf check;  // the -DLLAMA_CHECK build's violation bits
    DevBuf q_sums; // scratch of Eq. 2

    // bucketing scratch
    Workspace ws;  // the context's own scratch (llama_schedule, llama_schedule_async)
    // scoring kernel geometry (set by llama_set_profiles)
    int32_t min_vpl = 16, ipt = 2, stages = 1, score_grid = 0, score_chunk = 0, bucket_max_blocks = 0, dlat_cap = 0;
    int32_t score_per_sm = 0;  // persistent scoring CTAs per SM: 0 = as many as fit
    int32_t dlat_stage = kMaxDlatSmem;  // most distinct latencies of an op the scoring kernel stages
    size_t score_smem = 0;

    // staging for host-memory arguments of the blocking calls
    int64_t cap_stage = 0;
    DevBuf s_dag, s_opl, s_start, s_out, s_slack;
    unsigned long long *h_ctrl = nullptr;  // pinned copy of the control words

    int last_launches = 0;
    int32_t max_ncfg = 0;  // configurations of the largest op
    int32_t n_big_ops = 0;  // ops with more padded entries than dlat_cap
    int32_t n_cta_ops = 0;  // ops (bucket order) scored by whole CTAs; the rest by warp tiles
    int32_t count_pass = LLAMA_COUNT_PASS_AUTO;
    int32_t wait_tries = kMaxWaitTries;  // polls of a bucketing grid barrier (llama_set_wait_limit)
    int64_t direct_max = LLAMA_DIRECT_DEFAULT;  // small calls without bucketing (llama_set_direct_max)
    cudaEvent_t trace[LLAMA_TRACE_EVENTS] = {};
    bool tracing = false;

    // per-call statistics of the blocking scheduling call (llama_set_stats_file)
    FILE *stats = nullptr;
    int64_t stats_calls = 0;
    cudaEvent_t stats_ev[2] = {};

    // CUDA graph of the last untraced scheduling call (opts.use_graph): replayed
    // while the call's arguments and the context's buffers stay the same; `now`
    // is patched into the kernel that takes it.  Traced calls launch directly.
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaGraphNode_t g_bucket = nullptr;  // the captured kernel that takes `now`
    int g_now_nargs = 0;
    int g_launches = 2;  // kernel launches in the captured graph
    int64_t g_n_inv = -1, g_now = 0;
    const void *g_args[4] = {};

    void drop_graph() {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        gexec = nullptr;
        graph = nullptr;
        g_bucket = nullptr;
        g_n_inv = -1;
    }

    int fail(int code, const std::string &msg) {
        err = msg;
        return code;
    }
    void close_stats() {
        if (stats) fclose(stats);
        stats = nullptr;
        for (cudaEvent_t &e : stats_ev)
            if (e) cudaEventDestroy(e), e = nullptr;
    }
    int cuda_fail(cudaError_t e, const char *what) {
        err = std::string(what) + ": " + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? LLAMA_ENOMEM : LLAMA_ECUDA;
    }
};

#define LL_CUDA(ctx, call)                                   \
    do {                                                     \
        cudaError_t e__ = (call);                            \
        if (e__ != cudaSuccess) return (ctx)->cuda_fail(e__, #call); \
    } while (0)

namespace {

DevProblem make_problem(const llama_ctx *c) {
    DevProblem P{};
    P.n_dags = c->n_dags;
    P.n_ops = c->n_ops;
    P.n_hw = c->opts.n_hw;
    P.mode = c->opts.mode;
    P.dag_op_off = c->dag_op_off.as<int32_t>();
    P.row_ptr = c->row_ptr.as<int32_t>();
    P.col = c->col.as<int32_t>();
    P.slo = c->slo.as<int64_t>();
    P.dag_info = c->dag_info.as<int4>();
    P.cfg_off = c->cfg_off.as<int64_t>();
    P.hw_off = c->hw_off.as<int32_t>();
    P.lat = c->lat.as<int32_t>();
    P.cost = c->cost.as<int64_t>();
    P.ref_cfg = c->ref_cfg.as<int32_t>();
    P.batch = c->batch.as<int32_t>();
    P.res = c->res.as<int32_t>();
    P.res_total = c->res_total.as<int32_t>();
    P.pad_off = c->pad_off.as<int64_t>();
    P.seg_pad = c->seg_pad.as<int32_t>();
    P.lrb = c->lrb.as<uint16_t>();
    P.dlat = c->dlat.as<int32_t>();
    P.dlat_n = c->dlat_n.as<int32_t>();
    P.dpiv = c->dpiv.as<int32_t>();
    P.dpiv2 = c->dpiv2.p ? c->dpiv2.as<int32_t>() : nullptr;
    P.rf = c->rf.as<uint16_t>();
    P.df = c->df.as<uint16_t>();
    P.inv = c->inv.as<uint16_t>();
    P.fast = c->fast.as<int32_t>();
    P.op_order = c->op_order.as<int32_t>();
    P.max_npad = c->max_npad;
    P.n_big_ops = c->n_big_ops;
    P.n_cta_ops = c->n_cta_ops;
    // prefetch the encoded tables into L2 when they take at most half of it
    const int64_t tbl_bytes = (int64_t)(c->opts.mode == LLAMA_MODE_ALPHA ? 10 : 8) * c->n_pad;
    const bool pf = c->n_pad > 0 && tbl_bytes <= c->l2_bytes / 2;
    P.prefetch_rank_lines = pf ? (2 * c->n_pad + 127) / 128 : 0;
    P.prefetch_dlat_lines = pf ? (4 * c->n_pad + 127) / 128 : 0;
    P.ref_gidx = c->ref_gidx.as<int64_t>();
    P.ord_info = c->ord_info.as<int4>();
    P.ord_cbase = c->ord_cbase.as<int32_t>();
    P.dec = c->dec.as<int4>();
    P.dfast = c->dfast.as<int4>();
    P.stair = c->stair.as<uint16_t>();
    P.stair_off = c->stair_off.as<int64_t>();
    P.encode_only = nullptr;
    P.dag_pack = c->dag_pack.as<int32_t>();
    P.dag_pack_off = c->dag_pack_off.as<int64_t>();
    // arrays whose first touch starts a dependent chain: DAG structure, per-op
    // layout and the decode tables (lat, cost, inv) when they fit the budget
    {
        int a = 0;
        auto add = [&](const DevBuf &b) {
            if (a < kPfArrays && b.p && b.bytes) {
                P.pf_ptr[a] = static_cast<const char *>(b.p);
                P.pf_lines[a] = (int64_t)((b.bytes + 127) / 128);
                ++a;
            }
        };
        add(c->dag_op_off); add(c->slo); add(c->row_ptr); add(c->col); add(c->topo);
        add(c->lvl_off); add(c->dag_lvl); add(c->ref_gidx); add(c->op_order); add(c->pad_off);
        add(c->seg_pad); add(c->dlat_n); add(c->dfast); add(c->dpiv); add(c->ord_cbase);
        if (c->dec.bytes <= (size_t)c->l2_bytes / 4) add(c->dec);
        for (; a < kPfArrays; ++a) {
            P.pf_ptr[a] = nullptr;
            P.pf_lines[a] = 0;
        }
    }
    P.ref = c->ref.as<int64_t>();
    P.cp = c->cp.as<int64_t>();
    P.cp_magic = c->cp_magic.as<uint64_t>();
    P.q = c->q_dev.as<int64_t>();
    P.alpha_num = c->opts.alpha_num;
    P.alpha_den = c->opts.alpha_den;
    P.n_cfg = c->n_cfg;
    P.n_pad = c->n_pad;
    P.check = c->check.as<unsigned int>();
    P.wait_tries = c->wait_tries;
    return P;
}

BucketScratch make_scratch(const Workspace &w) {
    BucketScratch S{};
    S.cnt = w.cnt.as<int32_t>();
    S.ctrl = w.ctrl.as<unsigned long long>();
    S.status = S.ctrl + kCtrlWords;
    S.blk = reinterpret_cast<int4 *>(S.ctrl + kCtrlWords + kStatusWords);
    S.op_start = w.op_start.as<int32_t>();
    S.gop = w.gop.as<int32_t>();
    S.slot = w.slot.as<int32_t>();
    S.b_ent = w.b_ent.as<int2>();
    S.rbase = w.rbase.as<int64_t>();
    S.tiles = w.tiles.as<int4>();
    S.b_cnt = w.b_cnt.p ? w.b_cnt.as<uint16_t>() : nullptr;
    return S;
}

ContextView view_of(const llama_ctx *c) {
    ContextView v{};
    v.P = make_problem(c);
    v.topo = c->topo.as<int32_t>();
    v.lvl_off = c->lvl_off.as<int32_t>();
    v.dag_lvl = c->dag_lvl.as<int32_t>();
    v.n_dags = c->n_dags;
    v.n_ops = c->n_ops;
    v.n_hw = c->opts.n_hw;
    v.mode = c->opts.mode;
    v.device = c->opts.device;
    v.num_sms = c->num_sms;
    v.min_vpl = c->min_vpl;
    v.ipt = c->ipt;
    v.method = c->method;
    v.stages = c->stages;
    v.score_grid = c->score_grid;
    v.bucket_max_blocks = c->bucket_max_blocks;
    v.score_chunk = c->score_chunk;
    v.dlat_cap = c->dlat_cap;
    v.score_smem = c->score_smem;
    v.max_ncfg = c->max_ncfg;
    v.warp_tiles = c->n_cta_ops < c->n_ops;
    v.direct_max = c->method == LLAMA_METHOD_SCAN ? c->direct_max : 0;
    // the count pass: where some op may have more distinct latencies than the
    // scoring kernel stages, if asked for, or by default when such ops are at
    // least half of them (few invocations per table: the scoring kernel's own
    // searches would stand between the table copies)
    v.need_counts = c->max_ncfg > c->dlat_cap &&
                    (c->count_pass == LLAMA_COUNT_PASS_ON ||
                     (c->count_pass == LLAMA_COUNT_PASS_AUTO && 2 * (int64_t)c->n_big_ops >= c->n_ops));
    return v;
}

// Per-DAG packed structure for the critical-path pass (see DevProblem::dag_pack),
// built once both the DAGs and the profiles are known.
int build_dag_pack(llama_ctx *c) {
    if (!c->dags_set || !c->prof_set || c->n_ops_dag != c->n_ops) return LLAMA_OK;
    const int32_t nd = c->n_dags;
    std::vector<int64_t> off(nd + 1, 0);
    std::vector<int32_t> pk;
    for (int32_t d = 0; d < nd; ++d) {
        off[d] = (int64_t)pk.size();
        const int32_t lo = c->h_dag_op_off[d], hi = c->h_dag_op_off[d + 1], n = hi - lo;
        const int32_t e_lo = c->h_row_ptr[lo], ne = c->h_row_ptr[hi] - e_lo;
        const int32_t l_lo = c->h_dag_lvl[d], nl = c->h_dag_lvl[d + 1] - l_lo;
        const int64_t words = 4 + (int64_t)n + (n + 1) + ne + n + (nl + 1);
        if (n > kCpSmemOps || words > kCpPackWords) continue;  // empty: global-memory pass
        pk.push_back(lo);
        pk.push_back(n);
        pk.push_back(ne);
        pk.push_back(nl);
        for (int32_t v = lo; v < hi; ++v) pk.push_back((int32_t)c->h_ref_gidx[v]);
        for (int32_t v = lo; v <= hi; ++v) pk.push_back(c->h_row_ptr[v] - e_lo);
        for (int32_t e = 0; e < ne; ++e) pk.push_back(c->h_col[e_lo + e] - lo);
        for (int32_t v = lo; v < hi; ++v) pk.push_back(c->h_topo[v] - lo);
        for (int32_t l = 0; l <= nl; ++l) pk.push_back(c->h_lvl_off[l_lo + l] - lo);
    }
    off[nd] = (int64_t)pk.size();
    if (pk.empty()) pk.push_back(0);
    cudaError_t e;
    if ((e = c->dag_pack.alloc(4 * pk.size())) != cudaSuccess ||
        (e = cudaMemcpy(c->dag_pack.p, pk.data(), 4 * pk.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = c->dag_pack_off.alloc(8 * off.size())) != cudaSuccess ||
        (e = cudaMemcpy(c->dag_pack_off.p, off.data(), 8 * off.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return c->cuda_fail(e, "dag pack upload");
    return LLAMA_OK;
}

// The encodings of the profile tables (every op, or those P.encode_only flags):
// pads and fastest configuration, latency ranks and distinct latencies, probe
// lines, objective ranks, decode tables.  Enqueued on s.
cudaError_t encode_tables(llama_ctx *c, const DevProblem &P, cudaStream_t s) {
    const bool alpha = c->opts.mode == LLAMA_MODE_ALPHA;
    const int32_t n_ops = c->n_ops;
    k_encode_pad<<<n_ops, 256, 0, s>>>(P, c->lrb.as<uint16_t>(), c->rf.as<uint16_t>(),
                                       alpha ? c->df.as<uint16_t>() : nullptr, c->fast.as<int32_t>());
    k_encode_lat<<<n_ops, 1024, c->lat_smem, s>>>(P, c->lrb.as<uint16_t>(), c->dlat.as<int32_t>(),
                                                  c->dlat_n.as<int32_t>());
    k_encode_piv<<<(unsigned)((32 * (int64_t)n_ops + 255) / 256), 256, 0, s>>>(P, c->dpiv.as<int32_t>());
    if (c->dpiv2.p)
        k_encode_piv2<<<(unsigned)((1024 * (int64_t)n_ops + 255) / 256), 256, 0, s>>>(P, c->dpiv2.as<int32_t>());
    k_encode_rank<<<n_ops, 1024, c->sort_smem, s>>>(P, c->sort_cap, c->rf.as<uint16_t>(),
                                                    alpha ? c->df.as<uint16_t>() : nullptr, c->inv.as<uint16_t>());
    k_encode_dec<<<n_ops, 256, 0, s>>>(P, c->dec.as<int4>(), c->dfast.as<int4>());
    return cudaGetLastError();
}

// Staircase tables of the current profiles: H * (n_cfg + 1) 16-bit keys per op.
int build_stair(llama_ctx *c) {
    const int32_t n_ops = c->n_ops, H = c->opts.n_hw;
    std::vector<int64_t> off(n_ops + 1, 0);
    int32_t max_dn = 1;
    for (int32_t v = 0; v < n_ops; ++v) {
        off[v + 1] = off[v] + (int64_t)H * (c->h_ncfg[v] + 1);  // room for any distinct count
        max_dn = std::max(max_dn, c->h_ncfg[v]);
    }
    cudaError_t e;
    if ((e = c->stair.alloc(2 * (size_t)std::max<int64_t>(off[n_ops], 1))) != cudaSuccess ||
        (e = c->stair_off.alloc(8 * (size_t)(n_ops + 1))) != cudaSuccess ||
        (e = cudaMemcpy(c->stair_off.p, off.data(), 8 * (size_t)(n_ops + 1), cudaMemcpyHostToDevice)) != cudaSuccess)
        return c->cuda_fail(e, "staircase tables");
    const size_t smem = 2 * 4 * (size_t)(max_dn + 1);
    LL_CUDA(c, cudaFuncSetAttribute(k_encode_stair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const DevProblem P = make_problem(c);
    k_encode_stair<<<n_ops, 1024, smem, c->stream>>>(P, c->stair.as<uint16_t>());
    LL_CUDA(c, cudaGetLastError());
    LL_CUDA(c, cudaStreamSynchronize(c->stream));
    c->stair_ready = true;
    return LLAMA_OK;
}

// The context's own stream (blocking calls) waits for what is enqueued on s so far.
int order_context_after(llama_ctx *c, cudaStream_t s) {
    LL_CUDA(c, cudaEventRecord(c->order_ev, s));
    LL_CUDA(c, cudaStreamWaitEvent(c->stream, c->order_ev, 0));
    return LLAMA_OK;
}

int check_ready(llama_ctx *c) {
    if (!c->dags_set || !c->prof_set)
        return c->fail(LLAMA_ENOTREADY, "schedule called before llama_set_dags and llama_set_profiles");
    if (c->n_ops_dag != c->n_ops)
        return c->fail(LLAMA_EINVAL, "DAGs and profiles describe different numbers of operations");
    return LLAMA_OK;
}

// Grow workspace w for calls of up to n_inv invocations on the context's
// current operations (buffers move: the caller drops what points at them).
int ensure_ws(llama_ctx *c, Workspace &w, int64_t n_inv) {
    if (w.cap_ops < c->n_ops + 1) {
        const int32_t n = c->n_ops + 1;
        LL_CUDA(c, w.cnt.alloc(sizeof(int32_t) * kCntStride * n));
        LL_CUDA(c, w.ctrl.alloc(sizeof(unsigned long long) * (kCtrlWords + kStatusWords) +
                                sizeof(int4) * kMaxBucketBlocks));
        // counters and control words start at zero; every call leaves them so
        LL_CUDA(c, cudaMemset(w.cnt.p, 0, w.cnt.bytes));
        LL_CUDA(c, cudaMemset(w.ctrl.p, 0, w.ctrl.bytes));
        LL_CUDA(c, cudaDeviceSynchronize());  // before any stream of the caller uses them
        LL_CUDA(c, w.op_start.alloc(sizeof(int32_t) * n));
        w.cap_ops = n;
        w.cap_tiles = 0;
    }
    if (w.cap_inv < n_inv) {
        const int64_t n = std::max<int64_t>(n_inv, 1024);
        LL_CUDA(c, w.gop.alloc(sizeof(int32_t) * n));
        LL_CUDA(c, w.slot.alloc(sizeof(int32_t) * n));
        LL_CUDA(c, w.b_ent.alloc(sizeof(int2) * n));
        LL_CUDA(c, w.rbase.alloc(sizeof(int64_t) * n));
        LL_CUDA(c, w.b_cnt.alloc(sizeof(uint16_t) * LLAMA_MAX_HW * n));
        w.cap_inv = n;
        w.cap_tiles = 0;
    }
    const int64_t nt = max_tiles(w.cap_inv, c->n_ops);
    if (w.cap_tiles < nt) {
        LL_CUDA(c, w.tiles.alloc(2 * sizeof(int4) * nt));
        w.cap_tiles = nt;
    }
    return LLAMA_OK;
}

int ensure_scratch(llama_ctx *c, int64_t n_inv) {
    if (c->ws.cap_ops < c->n_ops + 1 || c->ws.cap_inv < n_inv) c->drop_graph();  // buffers move
    return ensure_ws(c, c->ws, n_inv);
}

int ensure_stage(llama_ctx *c, int64_t n_inv) {
    if (c->cap_stage >= n_inv) return LLAMA_OK;
    const int64_t n = std::max<int64_t>(n_inv, 1024);
    LL_CUDA(c, c->s_dag.alloc(sizeof(int32_t) * n));
    LL_CUDA(c, c->s_opl.alloc(sizeof(int32_t) * n));
    LL_CUDA(c, c->s_start.alloc(sizeof(int64_t) * n));
    LL_CUDA(c, c->s_out.alloc(sizeof(llama_decision) * n));
    LL_CUDA(c, c->s_slack.alloc(sizeof(int32_t) * n * c->opts.n_hw));
    c->cap_stage = n;
    return LLAMA_OK;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The address at which the current device's kernels can read p in place:
// device or managed memory, or page-locked host memory mapped into the device's
// address space (the kernels then read it over the host link, overlapped with
// their work); nullptr for pageable host memory, which must be copied.
const void *kernel_readable(const void *p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
    if (a.type == cudaMemoryTypeHost) return a.devicePointer;
    return nullptr;
}

int grid_for(const llama_ctx *c, int64_t n, int threads) {
    const int64_t want = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)c->num_sms * 16));
}

// The launch sequence of one scheduling call (all device pointers).
// Shared memory of the scoring kernel: per staging buffer, a chunk of latency
// ranks and objective ranks (plus rank differences in alpha mode) and the op's
// distinct latencies; then one count per (invocation, backend) for every group
// of the CTA (at most one group per thread).
// Shared-memory room for the distinct latencies of the largest op whose list
// has at most dlat_stage entries (none: every op is counted by the count pass
// or searched in global memory), and the ops whose padded tables exceed it
// (a prefix of the bucket order: they may need counts).
void apply_dlat_stage(llama_ctx *c) {
    int32_t cap = 0;
    for (int32_t v = 0; v < c->n_ops; ++v)
        if (c->h_dn[v] <= c->dlat_stage) cap = std::max(cap, c->h_dn[v]);
    c->dlat_cap = (cap + 3) / 4 * 4;
    c->n_big_ops = 0;
    for (int32_t v = 0; v < c->n_ops; ++v) c->n_big_ops += c->h_npad[v] > c->dlat_cap;
}

size_t score_smem_bytes(const llama_ctx *c) {
    const size_t tbl = ((size_t)c->score_chunk * (c->opts.mode == LLAMA_MODE_ALPHA ? 6 : 4) + 15) / 16 * 16;
    const size_t counts = (size_t)kScoreThreads * c->ipt * c->opts.n_hw * 2;
    const size_t cta = (size_t)c->stages * (tbl + 4 * (size_t)c->dlat_cap) + counts;
    // the warp phase reuses the same memory: one slice per warp
    return c->n_cta_ops < c->n_ops ? std::max(cta, (size_t)kScoreWarps * kWarpSlice) : cta;
}

// Default staging chunk: the largest padded table split into the fewest pieces
// of at most kMaxChunk entries plus the padding of its segments, as evenly as
// multiples of 8 allow (a table of 8,208 entries goes in two chunks of 4,104,
// not 4,096 + 4,096 + 16).
int32_t default_chunk(int32_t max_npad) {
    const int32_t cap = kMaxChunk + kVec * LLAMA_MAX_HW;
    const int32_t pieces = (max_npad + cap - 1) / cap;
    const int32_t per = (max_npad + pieces - 1) / pieces;
    return (per + kVec - 1) / kVec * kVec;
}

// Dynamic shared memory and persistent grid of the scoring kernel for the
// current profiles and tuning.
int configure_score(llama_ctx *c) {
    const void *fn = score_kernel(c->opts.mode, c->ipt, c->stages, c->n_cta_ops < c->n_ops);
    LL_CUDA(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->score_smem));
    int nb = 0;
    LL_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kScoreThreads, c->score_smem));
    if (c->score_per_sm > 0) nb = std::min(nb, c->score_per_sm);
    c->score_grid = c->num_sms * std::max(1, nb);
    return LLAMA_OK;
}

// Replace argument `index` of a captured kernel node by *value (same type).
template <class T>
cudaError_t patch_arg(cudaGraphExec_t exec, cudaGraphNode_t node, int n_args, int index, const T *value) {
    cudaKernelNodeParams p{};
    cudaError_t e = cudaGraphKernelNodeGetParams(node, &p);
    if (e != cudaSuccess) return e;
    if (!p.kernelParams || n_args > 16) return cudaErrorInvalidValue;
    void *args[16];
    for (int k = 0; k < n_args; ++k) args[k] = p.kernelParams[k];
    args[index] = const_cast<T *>(value);
    p.kernelParams = args;
    return cudaGraphExecKernelNodeSetParams(exec, node, &p);
}

int capture_graph(llama_ctx *c, int64_t n_inv, const int32_t *dag, const int32_t *op_local,
                  const int64_t *start, int64_t now, llama_decision *out) {
    c->drop_graph();
    const ContextView v = view_of(c);
    const BucketScratch S = make_scratch(c->ws);
    LL_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    const cudaError_t e = enqueue_schedule(v, S, n_inv, dag, op_local, start, now, out, c->cap_stream, nullptr);
    c->g_launches = schedule_launches(v, S, n_inv);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return c->cuda_fail(e, "capture enqueue_schedule");
    }
    LL_CUDA(c, e2);
    c->graph = g;
    LL_CUDA(c, cudaGraphInstantiate(&c->gexec, g, 0));
    size_t n = 0;
    LL_CUDA(c, cudaGraphGetNodes(g, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    LL_CUDA(c, cudaGraphGetNodes(g, nodes.data(), &n));
    for (cudaGraphNode_t node : nodes) {
        cudaGraphNodeType t;
        LL_CUDA(c, cudaGraphNodeGetType(node, &t));
        if (t == cudaGraphNodeTypeKernel) {
            cudaKernelNodeParams p{};
            LL_CUDA(c, cudaGraphKernelNodeGetParams(node, &p));
            // `now` is argument 5 of k_bucket (14 arguments), k_stair and k_direct_* (8)
            if (p.func == (void *)k_bucket) c->g_bucket = node, c->g_now_nargs = 14;
            if (p.func == (void *)k_stair || p.func == (void *)k_direct_cf || p.func == (void *)k_direct_al)
                c->g_bucket = node, c->g_now_nargs = 8;
        }
    }
    if (!c->g_bucket) return c->fail(LLAMA_ECUDA, "graph capture: kernel node not found");
    c->g_n_inv = n_inv;
    c->g_now = now;
    c->g_args[0] = dag;
    c->g_args[1] = op_local;
    c->g_args[2] = start;
    c->g_args[3] = out;
    return LLAMA_OK;
}

int launch_schedule(llama_ctx *c, int64_t n_inv, const int32_t *dag, const int32_t *op_local,
                    const int64_t *start, int64_t now, llama_decision *out, cudaStream_t s) {
    if (!c->opts.use_graph || c->tracing) {
        const ContextView v = view_of(c);
        const BucketScratch S = make_scratch(c->ws);
        LL_CUDA(c, enqueue_schedule(v, S, n_inv, dag, op_local, start, now, out, s,
                                    c->tracing ? c->trace : nullptr));
        c->last_launches = schedule_launches(v, S, n_inv);
        return LLAMA_OK;
    }
    const bool same = c->gexec && c->g_n_inv == n_inv && c->g_args[0] == dag &&
                      c->g_args[1] == op_local && c->g_args[2] == start && c->g_args[3] == out;
    if (!same) {
        const int rc = capture_graph(c, n_inv, dag, op_local, start, now, out);
        if (rc) return rc;
    }
    if (now != c->g_now) {
        LL_CUDA(c, patch_arg(c->gexec, c->g_bucket, c->g_now_nargs, 5, &now));
        c->g_now = now;
    }
    LL_CUDA(c, cudaGraphLaunch(c->gexec, s));
    c->last_launches = c->g_launches;
    return LLAMA_OK;
}

int check_inv_args(llama_ctx *c, int64_t n_inv, const void *a, const void *b, const void *d,
                   const void *o) {
    if (n_inv < 0 || n_inv > LLAMA_MAX_INV) return c->fail(LLAMA_EINVAL, "n_inv out of range");
    if (n_inv > 0 && (!a || !b || !d || !o)) return c->fail(LLAMA_EINVAL, "null invocation or output pointer");
    return LLAMA_OK;
}

}  // namespace

namespace llama {

int context_view(llama_ctx *c, ContextView *v) {
    const int rc = check_ready(c);
    if (rc) return rc;
    *v = view_of(c);
    return LLAMA_OK;
}

int context_fail(llama_ctx *c, int code, const char *msg) { return c->fail(code, msg); }

void context_set_launches(llama_ctx *c, int launches) { c->last_launches = launches; }

int context_ensure_stair(llama_ctx *c) {
    DeviceGuard g(c->opts.device);
    if (!c->prof_set) return c->fail(LLAMA_ENOTREADY, "staircase tables before llama_set_profiles");
    return c->stair_ready ? LLAMA_OK : build_stair(c);
}

}  // namespace llama

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" int llama_create(llama_ctx **out, const llama_opts *opts) {
    if (!out || !opts) return LLAMA_EINVAL;
    *out = nullptr;
    if (opts->mode != LLAMA_MODE_COST_FIRST && opts->mode != LLAMA_MODE_ALPHA) return LLAMA_EINVAL;
    if (opts->n_hw < 1 || opts->n_hw > LLAMA_MAX_HW) return LLAMA_EINVAL;
    if (opts->mode == LLAMA_MODE_ALPHA &&
        (opts->alpha_num < 1 || opts->alpha_num > LLAMA_MAX_ALPHA || opts->alpha_den < 1 ||
         opts->alpha_den > LLAMA_MAX_ALPHA))
        return LLAMA_EINVAL;
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess) {
        cudaGetLastError();
        return LLAMA_ECUDA;
    }
    if (opts->device < 0 || opts->device >= n_dev) return LLAMA_EINVAL;
    llama_ctx *c = new (std::nothrow) llama_ctx();
    if (!c) return LLAMA_ENOMEM;
    c->opts = *opts;
    DeviceGuard g(opts->device);
    int l2 = 0;
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, opts->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                               opts->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, opts->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->order_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(&c->h_ctrl, sizeof(unsigned long long) * kCtrlWords) != cudaSuccess ||
        c->q_dev.alloc(8 * LLAMA_MAX_HW) != cudaSuccess || c->q_sums.alloc(8 * LLAMA_MAX_HW) != cudaSuccess ||
        cudaMemset(c->q_dev.p, 0, 8 * LLAMA_MAX_HW) != cudaSuccess || c->check.alloc(16) != cudaSuccess ||
        cudaMemset(c->check.p, 0, 16) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return LLAMA_ECUDA;
    }
    c->l2_bytes = l2;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bucket, 256, 0) != cudaSuccess || nb < 1) {
        cudaGetLastError();
        llama_destroy(c);
        return LLAMA_ECUDA;
    }
    c->bucket_max_blocks = std::min(nb * c->num_sms, kMaxBucketBlocks);
    *out = c;
    return LLAMA_OK;
}

extern "C" void llama_destroy(llama_ctx *c) {
    if (!c) return;
    {
        DeviceGuard g(c->opts.device);
        if (c->stream) cudaStreamSynchronize(c->stream);
        c->drop_graph();
        if (c->stream) cudaStreamDestroy(c->stream);
        if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
        if (c->order_ev) cudaEventDestroy(c->order_ev);
        if (c->h_ctrl) cudaFreeHost(c->h_ctrl);
        c->close_stats();
        delete c;  // DevBuf destructors free device memory with the device current
    }
}

extern "C" const char *llama_last_error(llama_ctx *c) { return c ? c->err.c_str() : "null context"; }

extern "C" int llama_last_launch_count(llama_ctx *c) { return c ? c->last_launches : 0; }

extern "C" int llama_set_trace_events(llama_ctx *c, void *const *events, int32_t n_events) {
    if (!c) return LLAMA_EINVAL;
    if (n_events == 0) {
        c->tracing = false;
        return LLAMA_OK;
    }
    if (n_events != LLAMA_TRACE_EVENTS || !events)
        return c->fail(LLAMA_EINVAL, "set_trace_events: need LLAMA_TRACE_EVENTS event handles");
    for (int k = 0; k < LLAMA_TRACE_EVENTS; ++k) {
        if (!events[k]) return c->fail(LLAMA_EINVAL, "set_trace_events: null event");
        c->trace[k] = (cudaEvent_t)events[k];
    }
    c->tracing = true;
    return LLAMA_OK;
}

extern "C" int llama_set_dags(llama_ctx *c, int32_t n_dags, const int32_t *dag_op_off,
                              const int32_t *row_ptr, const int32_t *col, const int64_t *slo_us) {
    if (!c) return LLAMA_EINVAL;
    if (n_dags < 1 || !dag_op_off || !row_ptr || !slo_us)
        return c->fail(LLAMA_EINVAL, "set_dags: need n_dags >= 1 and non-null arrays");
    if (dag_op_off[0] != 0) return c->fail(LLAMA_EINVAL, "set_dags: dag_op_off[0] must be 0");
    for (int32_t d = 0; d < n_dags; ++d) {
        if (dag_op_off[d + 1] <= dag_op_off[d])
            return c->fail(LLAMA_EINVAL, "set_dags: every DAG needs at least one operation");
        if (slo_us[d] < 1 || slo_us[d] > INT32_MAX)
            return c->fail(LLAMA_EINVAL, "set_dags: slo_us out of 1..INT32_MAX");
    }
    const int32_t n_ops = dag_op_off[n_dags];
    if (row_ptr[0] != 0) return c->fail(LLAMA_EINVAL, "set_dags: row_ptr[0] must be 0");
    for (int32_t v = 0; v < n_ops; ++v)
        if (row_ptr[v + 1] < row_ptr[v]) return c->fail(LLAMA_EINVAL, "set_dags: row_ptr decreasing");
    const int32_t n_edges = row_ptr[n_ops];
    if (n_edges > 0 && !col) return c->fail(LLAMA_EINVAL, "set_dags: null col");
    std::vector<int32_t> owner(n_ops);
    for (int32_t d = 0; d < n_dags; ++d)
        for (int32_t v = dag_op_off[d]; v < dag_op_off[d + 1]; ++v) owner[v] = d;
    std::vector<int32_t> indeg(n_ops, 0);
    for (int32_t v = 0; v < n_ops; ++v)
        for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            const int32_t w = col[e];
            if (w < 0 || w >= n_ops || owner[w] != owner[v])
                return c->fail(LLAMA_EINVAL, "set_dags: edge leaves its DAG or is out of range");
            if (w == v) return c->fail(LLAMA_EINVAL, "set_dags: self-loop");
            ++indeg[w];
        }
    // Kahn order, then height above the sinks in reverse order
    std::vector<int32_t> order;
    order.reserve(n_ops);
    for (int32_t v = 0; v < n_ops; ++v)
        if (indeg[v] == 0) order.push_back(v);
    for (size_t h = 0; h < order.size(); ++h) {
        const int32_t v = order[h];
        for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e)
            if (--indeg[col[e]] == 0) order.push_back(col[e]);
    }
    if ((int32_t)order.size() != n_ops) return c->fail(LLAMA_EINVAL, "set_dags: the graph has a cycle");
    std::vector<int32_t> height(n_ops, 0);
    for (int32_t k = n_ops - 1; k >= 0; --k) {
        const int32_t v = order[k];
        int32_t hv = 0;
        for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) hv = std::max(hv, height[col[e]] + 1);
        height[v] = hv;
    }
    std::vector<int32_t> topo(n_ops), lvl_off, dag_lvl(n_dags + 1);
    for (int32_t d = 0; d < n_dags; ++d) {
        const int32_t lo = dag_op_off[d], hi = dag_op_off[d + 1];
        for (int32_t v = lo; v < hi; ++v) topo[v] = v;
        std::stable_sort(topo.begin() + lo, topo.begin() + hi,
                         [&](int32_t a, int32_t b) { return height[a] < height[b]; });
        dag_lvl[d] = (int32_t)lvl_off.size();
        for (int32_t p = lo; p < hi; ++p)
            if (p == lo || height[topo[p]] != height[topo[p - 1]]) lvl_off.push_back(p);
    }
    dag_lvl[n_dags] = (int32_t)lvl_off.size();
    lvl_off.push_back(n_ops);

    DeviceGuard g(c->opts.device);
    c->drop_graph();
    c->dags_set = false;
    auto up = [&](DevBuf &b, const void *h, size_t bytes) -> cudaError_t {
        cudaError_t e = b.alloc(bytes);
        if (e != cudaSuccess || bytes == 0) return e;
        return cudaMemcpy(b.p, h, bytes, cudaMemcpyHostToDevice);
    };
    std::vector<int32_t> info(4 * (size_t)n_dags);
    for (int32_t d = 0; d < n_dags; ++d) {
        info[4 * (size_t)d + 0] = dag_op_off[d];
        info[4 * (size_t)d + 1] = dag_op_off[d + 1];
        info[4 * (size_t)d + 2] = (int32_t)(uint32_t)((uint64_t)slo_us[d] & 0xFFFFFFFFu);
        info[4 * (size_t)d + 3] = (int32_t)(uint32_t)((uint64_t)slo_us[d] >> 32);
    }
    cudaError_t e;
    if ((e = up(c->dag_op_off, dag_op_off, 4 * (size_t)(n_dags + 1))) != cudaSuccess ||
        (e = up(c->dag_info, info.data(), 16 * (size_t)n_dags)) != cudaSuccess ||
        (e = up(c->row_ptr, row_ptr, 4 * (size_t)(n_ops + 1))) != cudaSuccess ||
        (e = up(c->col, col, 4 * (size_t)n_edges)) != cudaSuccess ||
        (e = up(c->slo, slo_us, 8 * (size_t)n_dags)) != cudaSuccess ||
        (e = up(c->topo, topo.data(), 4 * (size_t)n_ops)) != cudaSuccess ||
        (e = up(c->lvl_off, lvl_off.data(), 4 * lvl_off.size())) != cudaSuccess ||
        (e = up(c->dag_lvl, dag_lvl.data(), 4 * dag_lvl.size())) != cudaSuccess)
        return c->cuda_fail(e, "set_dags upload");
    c->n_dags = n_dags;
    c->n_ops_dag = n_ops;
    c->h_dag_op_off.assign(dag_op_off, dag_op_off + n_dags + 1);
    c->h_row_ptr.assign(row_ptr, row_ptr + n_ops + 1);
    c->h_col.assign(col, col + n_edges);
    c->h_topo = topo;
    c->h_lvl_off = lvl_off;
    c->h_dag_lvl = dag_lvl;
    c->dags_set = true;
    return build_dag_pack(c);
}

extern "C" int llama_set_profiles(llama_ctx *c, int32_t n_ops, const int64_t *cfg_off,
                                  const int32_t *hw_off, const int32_t *lat_us,
                                  const int64_t *cost_nd, const int32_t *ref_cfg,
                                  const int32_t *batch, const int32_t *res,
                                  const int32_t *res_total) {
    if (!c) return LLAMA_EINVAL;
    Range range("llama:set_profiles");
    const int H = c->opts.n_hw;
    const bool alpha = c->opts.mode == LLAMA_MODE_ALPHA;
    if (n_ops < 1 || !cfg_off || !hw_off || !lat_us || !cost_nd || !ref_cfg)
        return c->fail(LLAMA_EINVAL, "set_profiles: need n_ops >= 1 and non-null arrays");
    if (alpha && (!batch || !res || !res_total))
        return c->fail(LLAMA_EINVAL, "set_profiles: alpha mode needs batch, res and res_total");
    // resources are kept in either mode when given (Eq. 2's queueing time uses them)
    const bool with_res = batch && res && res_total;
    if (cfg_off[0] != 0) return c->fail(LLAMA_EINVAL, "set_profiles: cfg_off[0] must be 0");
    std::vector<int64_t> pad_off(n_ops + 1);
    std::vector<int32_t> seg_pad((size_t)n_ops * (H + 1));
    int32_t max_n = 0, max_npad = 0;
    pad_off[0] = 0;
    for (int32_t v = 0; v < n_ops; ++v) {
        const int64_t n = cfg_off[v + 1] - cfg_off[v];
        if (n < 1 || n > LLAMA_MAX_CFG)
            return c->fail(LLAMA_EINVAL, "set_profiles: configurations per op must be 1..8192");
        const int32_t *hw = hw_off + (size_t)v * (H + 1);
        if (hw[0] != 0 || hw[H] != n) return c->fail(LLAMA_EINVAL, "set_profiles: bad hw_off bounds");
        int32_t *sp = seg_pad.data() + (size_t)v * (H + 1);
        sp[0] = 0;
        for (int h = 0; h < H; ++h) {
            if (hw[h + 1] < hw[h]) return c->fail(LLAMA_EINVAL, "set_profiles: hw_off decreasing");
            sp[h + 1] = sp[h] + (int32_t)round_up(hw[h + 1] - hw[h], kVec);
        }
        if (ref_cfg[v] < 0 || ref_cfg[v] >= n)
            return c->fail(LLAMA_EINVAL, "set_profiles: ref_cfg out of range");
        pad_off[v + 1] = pad_off[v] + sp[H];
        max_n = std::max<int32_t>(max_n, (int32_t)n);
        max_npad = std::max<int32_t>(max_npad, sp[H]);
    }
    // bucket order of the ops: largest padded table first (stable), so the
    // scoring kernel's longest warps are launched first
    std::vector<int32_t> op_order(n_ops);
    for (int32_t v = 0; v < n_ops; ++v) op_order[v] = v;
    std::stable_sort(op_order.begin(), op_order.end(), [&](int32_t a, int32_t b) {
        return pad_off[a + 1] - pad_off[a] > pad_off[b + 1] - pad_off[b];
    });
    std::vector<int64_t> ref_gidx(n_ops);
    for (int32_t v = 0; v < n_ops; ++v) ref_gidx[v] = cfg_off[v] + ref_cfg[v];
    const int64_t n_cfg = cfg_off[n_ops];
    if (pad_off[n_ops] >= INT32_MAX) return c->fail(LLAMA_EINVAL, "set_profiles: padded tables too large");
    if (n_cfg >= INT32_MAX) return c->fail(LLAMA_EINVAL, "set_profiles: more than 2^31-1 configurations");
    for (int64_t x = 0; x < n_cfg; ++x) {
        if (lat_us[x] < 1 || lat_us[x] > INT32_MAX - 1)
            return c->fail(LLAMA_EINVAL, "set_profiles: latency out of 1..INT32_MAX-1");
        if (cost_nd[x] < 0) return c->fail(LLAMA_EINVAL, "set_profiles: negative cost");
        if (with_res && (batch[x] < 1 || batch[x] > LLAMA_MAX_ALPHA || res[x] < 1 || res[x] > LLAMA_MAX_ALPHA))
            return c->fail(LLAMA_EINVAL, "set_profiles: batch or res out of 1..65535");
    }
    if (with_res)
        for (int h = 0; h < H; ++h)
            if (res_total[h] < 1) return c->fail(LLAMA_EINVAL, "set_profiles: res_total must be >= 1");

    DeviceGuard g(c->opts.device);
    c->drop_graph();
    c->prof_set = false;
    const int64_t n_pad = pad_off[n_ops];
    auto up = [&](DevBuf &b, const void *h, size_t bytes) -> cudaError_t {
        cudaError_t e = b.alloc(bytes);
        if (e != cudaSuccess) return e;
        return cudaMemcpy(b.p, h, bytes, cudaMemcpyHostToDevice);
    };
    cudaError_t e;
    if ((e = up(c->cfg_off, cfg_off, 8 * (size_t)(n_ops + 1))) != cudaSuccess ||
        (e = up(c->hw_off, hw_off, 4 * (size_t)n_ops * (H + 1))) != cudaSuccess ||
        (e = up(c->lat, lat_us, 4 * (size_t)n_cfg)) != cudaSuccess ||
        (e = up(c->cost, cost_nd, 8 * (size_t)n_cfg)) != cudaSuccess ||
        (e = up(c->ref_cfg, ref_cfg, 4 * (size_t)n_ops)) != cudaSuccess ||
        (e = up(c->pad_off, pad_off.data(), 8 * (size_t)(n_ops + 1))) != cudaSuccess ||
        (e = up(c->seg_pad, seg_pad.data(), 4 * seg_pad.size())) != cudaSuccess ||
        (e = up(c->op_order, op_order.data(), 4 * (size_t)n_ops)) != cudaSuccess ||
        (e = up(c->ref_gidx, ref_gidx.data(), 8 * (size_t)n_ops)) != cudaSuccess ||
        (e = c->ord_info.alloc(16 * (size_t)n_ops)) != cudaSuccess ||
        (e = c->ord_cbase.alloc(4 * (size_t)n_ops)) != cudaSuccess ||
        (e = c->dec.alloc(16 * (alpha ? 2 : 1) * (size_t)n_cfg)) != cudaSuccess ||
        (e = c->dfast.alloc(16 * (size_t)n_ops)) != cudaSuccess ||
        (e = c->lrb.alloc(2 * (size_t)n_pad)) != cudaSuccess ||
        (e = c->dlat.alloc(4 * (size_t)n_pad)) != cudaSuccess ||
        (e = c->dlat_n.alloc(4 * (size_t)n_ops)) != cudaSuccess ||
        (e = c->dpiv.alloc(4 * 32 * (size_t)n_ops)) != cudaSuccess ||
        (e = c->rf.alloc(2 * (size_t)n_pad)) != cudaSuccess ||
        (e = c->inv.alloc(2 * 2 * (size_t)n_cfg)) != cudaSuccess ||
        (e = c->fast.alloc(4 * (size_t)n_ops)) != cudaSuccess ||
        (e = c->ref.alloc(8 * (size_t)n_ops)) != cudaSuccess ||
        (e = c->cp.alloc(8 * (size_t)n_ops)) != cudaSuccess ||
        (e = c->cp_magic.alloc(8 * (size_t)n_ops)) != cudaSuccess)
        return c->cuda_fail(e, "set_profiles upload");
    if (with_res) {
        if ((e = up(c->batch, batch, 4 * (size_t)n_cfg)) != cudaSuccess ||
            (e = up(c->res, res, 4 * (size_t)n_cfg)) != cudaSuccess ||
            (e = up(c->res_total, res_total, 4 * (size_t)H)) != cudaSuccess)
            return c->cuda_fail(e, "set_profiles upload");
    } else {
        c->batch.release();
        c->res.release();
        c->res_total.release();
    }
    if (alpha) {
        if ((e = c->df.alloc(2 * (size_t)n_pad)) != cudaSuccess) return c->cuda_fail(e, "set_profiles upload");
    } else {
        c->df.release();
    }
    // second-round probe lines (4 KB per op) where a search can use them: more
    // than 1,056 distinct latencies, so more than 1,024 configurations
    int64_t max_n_cfg = 0;
    for (int32_t v = 0; v < n_ops; ++v) max_n_cfg = std::max<int64_t>(max_n_cfg, cfg_off[v + 1] - cfg_off[v]);
    c->max_ncfg = (int32_t)max_n_cfg;
    if (max_n_cfg > 1024) {
        if ((e = c->dpiv2.alloc(4 * 1024 * (size_t)n_ops)) != cudaSuccess)
            return c->cuda_fail(e, "set_profiles upload");
    } else {
        c->dpiv2.release();
    }
    c->n_ops = n_ops;
    c->n_cfg = n_cfg;
    c->n_pad = n_pad;
    c->max_npad = max_npad;
    c->ws.cap_ops = 0;  // op count may have changed: re-size the per-op scratch

    c->max_n = max_n;
    c->sort_cap = 1;
    while (c->sort_cap < (alpha ? 2 * max_n : max_n)) c->sort_cap <<= 1;
    c->sort_smem = (size_t)c->sort_cap * 12;
    if (c->sort_smem > (size_t)c->max_smem_optin)
        return c->fail(LLAMA_EINVAL, "set_profiles: configuration space too large for one CTA sort");
    LL_CUDA(c, cudaFuncSetAttribute(k_encode_rank, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)c->sort_smem));
    int32_t lat_cap = 1;
    while (lat_cap < max_n) lat_cap <<= 1;
    c->lat_smem = (size_t)lat_cap * 8;
    LL_CUDA(c, cudaFuncSetAttribute(k_encode_lat, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->lat_smem));
    LL_CUDA(c, encode_tables(c, make_problem(c), c->stream));
    LL_CUDA(c, cudaStreamSynchronize(c->stream));
    {
        // bucket-order info per op: {op, vectors, padded offset, distinct latencies}
        std::vector<int32_t> dn(n_ops);
        LL_CUDA(c, cudaMemcpy(dn.data(), c->dlat_n.p, 4 * (size_t)n_ops, cudaMemcpyDeviceToHost));
        std::vector<int32_t> oi(4 * (size_t)n_ops);
        for (int32_t k2 = 0; k2 < n_ops; ++k2) {
            const int32_t v = op_order[k2];
            oi[4 * k2 + 0] = v;
            oi[4 * k2 + 1] = (int32_t)((pad_off[v + 1] - pad_off[v]) / kVec);
            oi[4 * k2 + 2] = (int32_t)pad_off[v];
            oi[4 * k2 + 3] = dn[v];
        }
        LL_CUDA(c, cudaMemcpy(c->ord_info.p, oi.data(), 16 * (size_t)n_ops, cudaMemcpyHostToDevice));
        std::vector<int32_t> cb(n_ops), pos(n_ops);
        for (int32_t k2 = 0; k2 < n_ops; ++k2) cb[k2] = (int32_t)cfg_off[op_order[k2]], pos[op_order[k2]] = k2;
        LL_CUDA(c, cudaMemcpy(c->ord_cbase.p, cb.data(), 4 * (size_t)n_ops, cudaMemcpyHostToDevice));
        LL_CUDA(c, c->ord_pos.alloc(4 * (size_t)n_ops));
        LL_CUDA(c, cudaMemcpy(c->ord_pos.p, pos.data(), 4 * (size_t)n_ops, cudaMemcpyHostToDevice));
        c->h_ncfg.resize(n_ops);
        for (int32_t v = 0; v < n_ops; ++v) c->h_ncfg[v] = (int32_t)(cfg_off[v + 1] - cfg_off[v]);
        // ops whose padded table fits a warp's slice are scored by warp tiles:
        // the end of the bucket order (largest tables first)
        c->n_cta_ops = 0;
        for (int32_t v = 0; v < n_ops; ++v) c->n_cta_ops += pad_off[v + 1] - pad_off[v] > warp_pad_of(c->opts.mode);
        c->h_dn = std::move(dn);
        c->h_npad.resize(n_ops);
        for (int32_t v = 0; v < n_ops; ++v) c->h_npad[v] = (int32_t)(pad_off[v + 1] - pad_off[v]);
        c->dlat_stage = kMaxDlatSmem;
        apply_dlat_stage(c);
    }
    c->stair_ready = false;

    // scoring kernel: stage tables in chunks of at most kMaxChunk entries, one
    // persistent CTA per resident slot
    c->score_chunk = default_chunk(max_npad);
    c->score_per_sm = 0;
    c->score_smem = score_smem_bytes(c);
    const int rc = configure_score(c);
    if (rc) return rc;
    c->h_ref_gidx = std::move(ref_gidx);
    c->prof_set = true;
    int rc2 = build_dag_pack(c);
    if (rc2 == LLAMA_OK && c->method == LLAMA_METHOD_STAIRCASE) rc2 = build_stair(c);
    return rc2;
}

extern "C" int llama_set_queue(llama_ctx *c, const int64_t *q_us) {
    if (!c) return LLAMA_EINVAL;
    if (!q_us) return c->fail(LLAMA_EINVAL, "set_queue: null q_us");
    for (int h = 0; h < c->opts.n_hw; ++h)
        if (q_us[h] < 0 || q_us[h] > INT32_MAX) return c->fail(LLAMA_EINVAL, "set_queue: q out of 0..INT32_MAX");
    int64_t q[LLAMA_MAX_HW] = {0};
    for (int h = 0; h < c->opts.n_hw; ++h) q[h] = q_us[h];
    DeviceGuard g(c->opts.device);
    // ordered after every call already enqueued on the legacy stream's side
    LL_CUDA(c, cudaDeviceSynchronize());
    LL_CUDA(c, cudaMemcpy(c->q_dev.p, q, sizeof(q), cudaMemcpyHostToDevice));
    return LLAMA_OK;
}

extern "C" int llama_queue_time(llama_ctx *c, int64_t n, const int32_t *dag, const int32_t *op_local,
                                const llama_decision *dec, int64_t *q_out, int32_t apply, void *stream) {
    if (!c) return LLAMA_EINVAL;
    if (n < 0 || (n > 0 && (!dag || !op_local || !dec))) return c->fail(LLAMA_EINVAL, "queue_time: bad arguments");
    int rc = check_ready(c);
    if (rc) return rc;
    if (!c->res.p || !c->res_total.p)
        return c->fail(LLAMA_EINVAL, "queue_time: the profiles carry no resources (res, res_total)");
    DeviceGuard g(c->opts.device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const DevProblem P = make_problem(c);
    LL_CUDA(c, cudaMemsetAsync(c->q_sums.p, 0, c->q_sums.bytes, s));
    if (n > 0)
        k_queue_sum<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(
            P, n, dag, op_local, dec, c->q_sums.as<unsigned long long>());
    k_queue_finish<<<1, 32, 0, s>>>(P, c->q_sums.as<unsigned long long>(), q_out,
                                     apply ? c->q_dev.as<int64_t>() : nullptr);
    LL_CUDA(c, cudaGetLastError());
    return apply ? order_context_after(c, s) : LLAMA_OK;
}

extern "C" int llama_set_tuning(llama_ctx *c, int32_t lanes_min_vectors, int32_t inv_per_thread,
                                int32_t chunk_entries, int32_t stages) {
    if (!c) return LLAMA_EINVAL;
    if (lanes_min_vectors < 1 || lanes_min_vectors > 1024)
        return c->fail(LLAMA_EINVAL, "set_tuning: lanes_min_vectors out of 1..1024");
    if (inv_per_thread != 1 && inv_per_thread != 2 && inv_per_thread != 4)
        return c->fail(LLAMA_EINVAL, "set_tuning: inv_per_thread must be 1, 2 or 4");
    if (chunk_entries < 0 || chunk_entries > LLAMA_MAX_CFG + kVec * LLAMA_MAX_HW || chunk_entries % kVec)
        return c->fail(LLAMA_EINVAL, "set_tuning: chunk_entries must be a multiple of 8 in 0..8256");
    if (stages != 1 && stages != 2) return c->fail(LLAMA_EINVAL, "set_tuning: stages must be 1 or 2");
    if (!c->prof_set) return c->fail(LLAMA_ENOTREADY, "set_tuning: set the profiles first");
    DeviceGuard g(c->opts.device);
    c->drop_graph();
    c->min_vpl = lanes_min_vectors;
    c->ipt = inv_per_thread;
    c->stages = stages;
    c->score_chunk = chunk_entries ? std::min<int32_t>(chunk_entries, c->max_npad) : default_chunk(c->max_npad);
    c->score_smem = score_smem_bytes(c);
    return configure_score(c);
}

extern "C" int llama_set_dlat_stage(llama_ctx *c, int32_t max_entries) {
    if (!c) return LLAMA_EINVAL;
    if (max_entries < 1 || max_entries > LLAMA_MAX_CFG)
        return c->fail(LLAMA_EINVAL, "set_dlat_stage: max_entries out of 1..8192");
    if (!c->prof_set) return c->fail(LLAMA_ENOTREADY, "set_dlat_stage: set the profiles first");
    DeviceGuard g(c->opts.device);
    c->drop_graph();
    c->dlat_stage = max_entries;
    apply_dlat_stage(c);
    c->score_smem = score_smem_bytes(c);
    return configure_score(c);
}

extern "C" int llama_set_score_occupancy(llama_ctx *c, int32_t ctas_per_sm) {
    if (!c) return LLAMA_EINVAL;
    if (ctas_per_sm < 0 || ctas_per_sm > 32)
        return c->fail(LLAMA_EINVAL, "set_score_occupancy: ctas_per_sm out of 0..32");
    if (!c->prof_set) return c->fail(LLAMA_ENOTREADY, "set_score_occupancy: set the profiles first");
    DeviceGuard g(c->opts.device);
    c->drop_graph();
    c->score_per_sm = ctas_per_sm;
    return configure_score(c);
}

extern "C" int llama_set_count_pass(llama_ctx *c, int32_t mode) {
    if (!c) return LLAMA_EINVAL;
    if (mode != LLAMA_COUNT_PASS_AUTO && mode != LLAMA_COUNT_PASS_ON && mode != LLAMA_COUNT_PASS_OFF)
        return c->fail(LLAMA_EINVAL, "set_count_pass: mode must be LLAMA_COUNT_PASS_AUTO, _ON or _OFF");
    if (mode != c->count_pass) {
        DeviceGuard g(c->opts.device);
        c->drop_graph();  // the captured launch sequence changes
        c->count_pass = mode;
    }
    return LLAMA_OK;
}

extern "C" int llama_check_build(void) {
#ifdef LLAMA_CHECK
    return 1;
#else
    return 0;
#endif
}

extern "C" int llama_check_word(llama_ctx *c, uint32_t *bits, int32_t clear) {
    if (!c || !bits) return LLAMA_EINVAL;
    DeviceGuard g(c->opts.device);
    LL_CUDA(c, cudaDeviceSynchronize());
    LL_CUDA(c, cudaMemcpy(bits, c->check.p, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    if (clear) LL_CUDA(c, cudaMemset(c->check.p, 0, sizeof(uint32_t)));
    return LLAMA_OK;
}

extern "C" int llama_set_stats_file(llama_ctx *c, const char *path) {
    if (!c) return LLAMA_EINVAL;
    DeviceGuard g(c->opts.device);
    c->close_stats();
    if (!path || !*path) return LLAMA_OK;
    c->stats = fopen(path, "a");
    if (!c->stats) return c->fail(LLAMA_EINVAL, std::string("set_stats_file: cannot open ") + path);
    LL_CUDA(c, cudaEventCreate(&c->stats_ev[0]));
    LL_CUDA(c, cudaEventCreate(&c->stats_ev[1]));
    return LLAMA_OK;
}

extern "C" int llama_set_wait_limit(llama_ctx *c, int32_t tries) {
    if (!c) return LLAMA_EINVAL;
    if (tries < 0 || tries > kMaxWaitTries)
        return c->fail(LLAMA_EINVAL, "set_wait_limit: tries must be in 0..LLAMA_WAIT_LIMIT_DEFAULT");
    if (tries != c->wait_tries) {
        DeviceGuard g(c->opts.device);
        c->drop_graph();  // the limit is a kernel argument of the captured launches
        c->wait_tries = tries;
    }
    return LLAMA_OK;
}

extern "C" int llama_set_direct_max(llama_ctx *c, int64_t n_inv) {
    if (!c) return LLAMA_EINVAL;
    if (n_inv < 0 || n_inv > LLAMA_DIRECT_LIMIT)
        return c->fail(LLAMA_EINVAL, "set_direct_max: n_inv must be in 0..LLAMA_DIRECT_LIMIT");
    if (n_inv != c->direct_max) {
        DeviceGuard g(c->opts.device);
        c->drop_graph();  // the captured launch sequence changes
        c->direct_max = n_inv;
    }
    return LLAMA_OK;
}

extern "C" int llama_set_method(llama_ctx *c, int32_t method) {
    if (!c) return LLAMA_EINVAL;
    if (method != LLAMA_METHOD_SCAN && method != LLAMA_METHOD_STAIRCASE)
        return c->fail(LLAMA_EINVAL, "set_method: method must be LLAMA_METHOD_SCAN or LLAMA_METHOD_STAIRCASE");
    DeviceGuard g(c->opts.device);
    c->drop_graph();
    c->method = method;
    if (method == LLAMA_METHOD_STAIRCASE && c->prof_set && !c->stair_ready) return build_stair(c);
    return LLAMA_OK;
}

extern "C" int llama_feedback(llama_ctx *c, int64_t n, const int32_t *op, const int32_t *cfg,
                              const int32_t *lat_us, const int64_t *cost_nd, int32_t beta_num, int32_t beta_den,
                              int64_t *rejected, void *stream) {
    if (!c) return LLAMA_EINVAL;
    Range range("llama:feedback");
    if (n < 0 || n >= INT32_MAX || (n > 0 && (!op || !cfg || !lat_us || !cost_nd)))
        return c->fail(LLAMA_EINVAL, "feedback: bad arguments");
    if (beta_den < 1 || beta_den > LLAMA_MAX_ALPHA || beta_num < 0 || beta_num > beta_den)
        return c->fail(LLAMA_EINVAL, "feedback: need 0 <= beta_num <= beta_den <= 65535, beta_den >= 1");
    int rc = check_ready(c);
    if (rc) return rc;
    DeviceGuard g(c->opts.device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n == 0) return LLAMA_OK;
    const size_t cap = 4 * (size_t)n;
    if (c->fb_keys.bytes < cap) {
        LL_CUDA(c, c->fb_keys.alloc(cap));
        LL_CUDA(c, c->fb_idx.alloc(cap));
        LL_CUDA(c, c->fb_keys2.alloc(cap));
        LL_CUDA(c, c->fb_idx2.alloc(cap));
    }
    if (c->fb_touched.bytes < (size_t)c->n_ops) LL_CUDA(c, c->fb_touched.alloc((size_t)c->n_ops));
    if (!c->fb_rejected.p) LL_CUDA(c, c->fb_rejected.alloc(8));
    size_t tmp = 0;
    LL_CUDA(c, cub::DeviceRadixSort::SortPairs(nullptr, tmp, c->fb_keys.as<int32_t>(), c->fb_keys2.as<int32_t>(),
                                               c->fb_idx.as<int32_t>(), c->fb_idx2.as<int32_t>(), (int)n, 0, 32, s));
    if (c->fb_tmp.bytes < tmp) LL_CUDA(c, c->fb_tmp.alloc(tmp));
    DevProblem P = make_problem(c);
    LL_CUDA(c, cudaMemsetAsync(c->fb_touched.p, 0, (size_t)c->n_ops, s));
    LL_CUDA(c, cudaMemsetAsync(c->fb_rejected.p, 0, 8, s));
    const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
    k_feedback_keys<<<grid, 256, 0, s>>>(P, n, op, cfg, lat_us, cost_nd, c->fb_keys.as<int32_t>(),
                                         c->fb_idx.as<int32_t>(), c->fb_rejected.as<unsigned long long>());
    LL_CUDA(c, cub::DeviceRadixSort::SortPairs(c->fb_tmp.p, tmp, c->fb_keys.as<int32_t>(), c->fb_keys2.as<int32_t>(),
                                               c->fb_idx.as<int32_t>(), c->fb_idx2.as<int32_t>(), (int)n, 0, 32, s));
    k_feedback_apply<<<grid, 256, 0, s>>>(P, n, c->fb_keys2.as<int32_t>(), c->fb_idx2.as<int32_t>(), op, lat_us,
                                          cost_nd, beta_num, beta_den, c->lat.as<int32_t>(), c->cost.as<int64_t>(),
                                          c->fb_touched.as<uint8_t>());
    // rebuild the encodings of the touched ops, on the device
    P.encode_only = c->fb_touched.as<uint8_t>();
    LL_CUDA(c, encode_tables(c, P, s));
    k_refresh_order<<<(c->n_ops + 255) / 256, 256, 0, s>>>(P, c->ord_pos.as<int32_t>(), c->ord_info.as<int4>());
    if (c->stair_ready) {
        const size_t smem = 2 * 4 * (size_t)(c->max_n + 1);
        k_encode_stair<<<c->n_ops, 1024, smem, s>>>(P, c->stair.as<uint16_t>());
    }
    if (rejected) LL_CUDA(c, cudaMemcpyAsync(rejected, c->fb_rejected.p, 8, cudaMemcpyDeviceToDevice, s));
    LL_CUDA(c, cudaGetLastError());
    return order_context_after(c, s);
}

extern "C" int llama_backend_objectives(llama_ctx *c, int64_t n_inv, const int32_t *dag, const int32_t *op_local,
                                        const int64_t *start_us, int64_t now_us, int64_t *obj_min, void *stream) {
    if (!c) return LLAMA_EINVAL;
    int rc = check_inv_args(c, n_inv, dag, op_local, start_us, obj_min);
    if (rc) return rc;
    if ((rc = check_ready(c))) return rc;
    if (!c->res.p || !c->batch.p || !c->res_total.p)
        return c->fail(LLAMA_EINVAL, "backend_objectives: Eq. 1 needs batch, res and res_total in the profiles");
    if (c->opts.alpha_num < 0 || c->opts.alpha_num > LLAMA_MAX_ALPHA || c->opts.alpha_den < 1 ||
        c->opts.alpha_den > LLAMA_MAX_ALPHA)
        return c->fail(LLAMA_EINVAL, "backend_objectives: the context's alpha is not usable (llama_opts)");
    if (n_inv == 0) return LLAMA_OK;
    DeviceGuard g(c->opts.device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const ContextView v = view_of(c);
    k_critical_paths<<<std::max(1, (v.n_dags + 7) / 8), 256, 0, s>>>(v.P, v.topo, v.lvl_off, v.dag_lvl);
    k_backend_obj<<<(unsigned)((n_inv * 32 + 255) / 256), 256, 0, s>>>(v.P, n_inv, dag, op_local, start_us, now_us,
                                                                       obj_min);
    LL_CUDA(c, cudaGetLastError());
    return LLAMA_OK;
}

extern "C" int llama_commit_order(llama_ctx *c, int64_t n, const int32_t *dag, const int32_t *op_local,
                                  const llama_decision *dec, const int64_t *obj_min, int32_t *order,
                                  double *affinity, void *stream) {
    if (!c) return LLAMA_EINVAL;
    if (n < 0 || n >= INT32_MAX || (n > 0 && (!dag || !op_local || !dec || !obj_min || !order)))
        return c->fail(LLAMA_EINVAL, "commit_order: bad arguments");
    int rc = check_ready(c);
    if (rc) return rc;
    if (n == 0) return LLAMA_OK;
    DeviceGuard g(c->opts.device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t need = 8 * (size_t)n;
    if (c->co_aff.bytes < need) {
        LL_CUDA(c, c->co_aff.alloc(need));
        LL_CUDA(c, c->co_aff2.alloc(need));
        LL_CUDA(c, c->co_lam.alloc(4 * (size_t)n));
        LL_CUDA(c, c->co_lam2.alloc(4 * (size_t)n));
        LL_CUDA(c, c->co_idx.alloc(4 * (size_t)n));
        LL_CUDA(c, c->co_idx2.alloc(4 * (size_t)n));
    }
    const DevProblem P = make_problem(c);
    k_commit_keys<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(
        P, n, dag, op_local, dec, obj_min, c->co_aff.as<uint64_t>(), c->co_lam.as<uint32_t>(), c->co_idx.as<int32_t>(),
        affinity);
    // two stable sorts: by affinity (descending keys), then by backend
    size_t t1 = 0, t2 = 0;
    LL_CUDA(c, cub::DeviceRadixSort::SortPairs(nullptr, t1, c->co_aff.as<uint64_t>(), c->co_aff2.as<uint64_t>(),
                                               c->co_idx.as<int32_t>(), c->co_idx2.as<int32_t>(), (int)n, 0, 64, s));
    LL_CUDA(c, cub::DeviceRadixSort::SortPairs(nullptr, t2, c->co_lam.as<uint32_t>(), c->co_lam2.as<uint32_t>(),
                                               c->co_idx2.as<int32_t>(), order, (int)n, 0, 8, s));
    if (c->co_tmp.bytes < std::max(t1, t2)) LL_CUDA(c, c->co_tmp.alloc(std::max(t1, t2)));
    LL_CUDA(c, cub::DeviceRadixSort::SortPairs(c->co_tmp.p, t1, c->co_aff.as<uint64_t>(), c->co_aff2.as<uint64_t>(),
                                               c->co_idx.as<int32_t>(), c->co_idx2.as<int32_t>(), (int)n, 0, 64, s));
    // the backend of each entry in affinity order, then the stable sort by it
    k_gather_u32<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(
        n, c->co_lam.as<uint32_t>(), c->co_idx2.as<int32_t>(), c->co_lam2.as<uint32_t>());
    LL_CUDA(c, cub::DeviceRadixSort::SortPairs(c->co_tmp.p, t2, c->co_lam2.as<uint32_t>(), c->co_lam.as<uint32_t>(),
                                               c->co_idx2.as<int32_t>(), order, (int)n, 0, 8, s));
    LL_CUDA(c, cudaGetLastError());
    return LLAMA_OK;
}

extern "C" int llama_get_profiles(llama_ctx *c, int32_t *lat_us, int64_t *cost_nd) {
    if (!c) return LLAMA_EINVAL;
    int rc = check_ready(c);
    if (rc) return rc;
    DeviceGuard g(c->opts.device);
    LL_CUDA(c, cudaDeviceSynchronize());
    if (lat_us) LL_CUDA(c, cudaMemcpy(lat_us, c->lat.p, 4 * (size_t)c->n_cfg, cudaMemcpyDeviceToHost));
    if (cost_nd) LL_CUDA(c, cudaMemcpy(cost_nd, c->cost.p, 8 * (size_t)c->n_cfg, cudaMemcpyDeviceToHost));
    return LLAMA_OK;
}

extern "C" int llama_reserve(llama_ctx *c, int64_t max_inv) {
    if (!c) return LLAMA_EINVAL;
    if (max_inv < 0 || max_inv > LLAMA_MAX_INV) return c->fail(LLAMA_EINVAL, "reserve: out of range");
    int rc = check_ready(c);
    if (rc) return rc;
    DeviceGuard g(c->opts.device);
    return ensure_scratch(c, max_inv);
}

struct llama_ws {
    Workspace w;
    llama_ctx *ctx = nullptr;
    int device = 0;
    DevBuf out_stage;  // decisions of a call whose output is page-locked host memory
    int32_t inputs = LLAMA_WS_INPUTS_IN_PLACE;
    DevBuf in_dag, in_opl, in_start;  // copies of page-locked host inputs (LLAMA_WS_INPUTS_COPY)
};

extern "C" int llama_ws_create(llama_ctx *c, int64_t max_inv, llama_ws **out) {
    if (!c || !out) return LLAMA_EINVAL;
    *out = nullptr;
    if (max_inv < 1 || max_inv > LLAMA_MAX_INV) return c->fail(LLAMA_EINVAL, "ws_create: max_inv out of range");
    int rc = check_ready(c);
    if (rc) return rc;
    DeviceGuard g(c->opts.device);
    llama_ws *ws = new llama_ws();
    ws->ctx = c;
    ws->device = c->opts.device;
    if ((rc = ensure_ws(c, ws->w, max_inv))) {
        delete ws;
        return rc;
    }
    *out = ws;
    return LLAMA_OK;
}

extern "C" void llama_ws_destroy(llama_ws *ws) {
    if (!ws) return;
    DeviceGuard g(ws->device);
    delete ws;
}

extern "C" int llama_schedule_ws_async(llama_ctx *c, llama_ws *ws, int64_t n_inv, const int32_t *dag,
                                       const int32_t *op_local, const int64_t *start_us, int64_t now_us,
                                       llama_decision *out, void *stream) {
    if (!c || !ws) return LLAMA_EINVAL;
    if (ws->ctx != c) return c->fail(LLAMA_EINVAL, "schedule_ws: workspace of another context");
    int rc = check_inv_args(c, n_inv, dag, op_local, start_us, out);
    if (rc) return rc;
    if ((rc = check_ready(c))) return rc;
    if (n_inv == 0) return LLAMA_OK;
    if (n_inv > ws->w.cap_inv) return c->fail(LLAMA_EINVAL, "schedule_ws: more invocations than the workspace holds");
    if (ws->w.cap_ops < c->n_ops + 1 || ws->w.cap_tiles < max_tiles(n_inv, c->n_ops))
        return c->fail(LLAMA_EINVAL, "schedule_ws: workspace sized for fewer operations (profiles changed)");
    DeviceGuard g(c->opts.device);
    // device or page-locked host memory: inputs read in place, decisions for a
    // host output written to the workspace's staging buffer and copied back
    // on the stream
    const void *rd = kernel_readable(dag), *ro = kernel_readable(op_local), *rs = kernel_readable(start_us);
    if (!rd || !ro || !rs)
        return c->fail(LLAMA_EINVAL, "schedule_ws: inputs must be device or page-locked host memory");
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (ws->inputs == LLAMA_WS_INPUTS_COPY) {
        // host inputs copied into the workspace by the copy engine on the stream
        const int64_t cap = ws->w.cap_inv;
        struct In {
            const void *src, **dst;
            DevBuf *buf;
            size_t elem;
        } ins[3] = {{dag, &rd, &ws->in_dag, 4}, {op_local, &ro, &ws->in_opl, 4}, {start_us, &rs, &ws->in_start, 8}};
        for (In &in : ins) {
            if (is_device_ptr(in.src)) continue;
            if (in.buf->bytes < in.elem * (size_t)cap) LL_CUDA(c, in.buf->alloc(in.elem * (size_t)cap));
            LL_CUDA(c, cudaMemcpyAsync(in.buf->p, in.src, in.elem * (size_t)n_inv, cudaMemcpyHostToDevice, s));
            *in.dst = in.buf->p;
        }
    }
    const bool outd = is_device_ptr(out);
    if (!outd) {
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, out) != cudaSuccess || a.type != cudaMemoryTypeHost) {
            cudaGetLastError();
            return c->fail(LLAMA_EINVAL, "schedule_ws: out must be device or page-locked host memory");
        }
        if (ws->out_stage.bytes < sizeof(llama_decision) * (size_t)ws->w.cap_inv)
            LL_CUDA(c, ws->out_stage.alloc(sizeof(llama_decision) * (size_t)ws->w.cap_inv));
    }
    llama_decision *d_out = outd ? out : ws->out_stage.as<llama_decision>();
    const ContextView v = view_of(c);
    LL_CUDA(c, enqueue_schedule(v, make_scratch(ws->w), n_inv, static_cast<const int32_t *>(rd),
                                static_cast<const int32_t *>(ro), static_cast<const int64_t *>(rs), now_us, d_out,
                                s, nullptr));
    if (!outd) LL_CUDA(c, cudaMemcpyAsync(out, d_out, sizeof(llama_decision) * n_inv, cudaMemcpyDeviceToHost, s));
    return LLAMA_OK;
}

extern "C" int llama_ws_set_inputs(llama_ws *ws, int32_t mode) {
    if (!ws || (mode != LLAMA_WS_INPUTS_IN_PLACE && mode != LLAMA_WS_INPUTS_COPY)) return LLAMA_EINVAL;
    ws->inputs = mode;
    return LLAMA_OK;
}

extern "C" int llama_ws_status(llama_ws *ws, int64_t *invalid, int32_t *timeout) {
    if (!ws) return LLAMA_EINVAL;
    DeviceGuard g(ws->device);
    unsigned long long st[kStatusWords] = {0, 0};
    if (cudaMemcpy(st, ws->w.ctrl.as<unsigned long long>() + kCtrlWords, sizeof(st), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
        return LLAMA_ECUDA;
    if (invalid) *invalid = (int64_t)st[0];
    if (timeout) *timeout = st[1] ? 1 : 0;
    return LLAMA_OK;
}

extern "C" int llama_schedule_async(llama_ctx *c, int64_t n_inv, const int32_t *dag,
                                    const int32_t *op_local, const int64_t *start_us, int64_t now_us,
                                    llama_decision *out, void *stream) {
    if (!c) return LLAMA_EINVAL;
    Range range("llama:schedule_async");
    int rc = check_inv_args(c, n_inv, dag, op_local, start_us, out);
    if (rc) return rc;
    if ((rc = check_ready(c))) return rc;
    if (n_inv == 0) return LLAMA_OK;
    DeviceGuard g(c->opts.device);
    if ((rc = ensure_scratch(c, n_inv))) return rc;
    return launch_schedule(c, n_inv, dag, op_local, start_us, now_us, out, (cudaStream_t)stream);
}

extern "C" int llama_schedule(llama_ctx *c, int64_t n_inv, const int32_t *dag, const int32_t *op_local,
                              const int64_t *start_us, int64_t now_us, llama_decision *out) {
    if (!c) return LLAMA_EINVAL;
    Range range("llama:schedule");
    const auto t_call = std::chrono::steady_clock::now();
    int rc = check_inv_args(c, n_inv, dag, op_local, start_us, out);
    if (rc) return rc;
    if ((rc = check_ready(c))) return rc;
    if (n_inv == 0) return LLAMA_OK;
    DeviceGuard g(c->opts.device);
    if ((rc = ensure_scratch(c, n_inv))) return rc;
    // inputs in device memory or page-locked host memory are read in place
    // (reading over the host link from the kernels measured faster than a copy
    // engine transfer followed by the kernels); pageable ones are copied; the
    // decisions are written to device memory and copied back (scattered writes
    // of 24-byte records over the host link are slow)
    const void *rd = kernel_readable(dag), *ro = kernel_readable(op_local), *rs = kernel_readable(start_us);
    const bool outd = is_device_ptr(out);
    if (!(rd && ro && rs && outd) && (rc = ensure_stage(c, n_inv))) return rc;
    cudaStream_t s = c->stream;
    const int32_t *d_dag = rd ? static_cast<const int32_t *>(rd) : c->s_dag.as<int32_t>();
    const int32_t *d_opl = ro ? static_cast<const int32_t *>(ro) : c->s_opl.as<int32_t>();
    const int64_t *d_start = rs ? static_cast<const int64_t *>(rs) : c->s_start.as<int64_t>();
    llama_decision *d_out = outd ? out : c->s_out.as<llama_decision>();
    if (!rd) LL_CUDA(c, cudaMemcpyAsync((void *)d_dag, dag, 4 * n_inv, cudaMemcpyHostToDevice, s));
    if (!ro) LL_CUDA(c, cudaMemcpyAsync((void *)d_opl, op_local, 4 * n_inv, cudaMemcpyHostToDevice, s));
    if (!rs) LL_CUDA(c, cudaMemcpyAsync((void *)d_start, start_us, 8 * n_inv, cudaMemcpyHostToDevice, s));
    if (c->stats) LL_CUDA(c, cudaEventRecord(c->stats_ev[0], s));
    if ((rc = launch_schedule(c, n_inv, d_dag, d_opl, d_start, now_us, d_out, s))) return rc;
    if (c->stats) LL_CUDA(c, cudaEventRecord(c->stats_ev[1], s));
    if (!outd) LL_CUDA(c, cudaMemcpyAsync(out, d_out, sizeof(llama_decision) * n_inv, cudaMemcpyDeviceToHost, s));
    LL_CUDA(c, cudaMemcpyAsync(c->h_ctrl, c->ws.ctrl.as<unsigned long long>() + kCtrlWords,
                               sizeof(unsigned long long) * kStatusWords, cudaMemcpyDeviceToHost, s));
    LL_CUDA(c, cudaStreamSynchronize(s));
    if (c->stats) {
        // one JSON object per line: the call's size, its kernels, what it found
        // and how long it took on the device (kernels only) and on the host (whole call)
        float dev_ms = 0.f;
        cudaEventElapsedTime(&dev_ms, c->stats_ev[0], c->stats_ev[1]);
        const double host_us =
            std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t_call).count();
        // with the decisions (and the invocations) in host memory: how many met
        // their target, and how many configurations the decided ones scored
        char feas[32] = "null", scored[32] = "null", cps[32] = "null";
        if (!outd) {
            int64_t nf = 0;
            for (int64_t i = 0; i < n_inv; ++i) nf += (out[i].flags & LLAMA_FLAG_FEASIBLE) != 0;
            snprintf(feas, sizeof feas, "%lld", (long long)nf);
            if (!is_device_ptr(dag) && !is_device_ptr(op_local)) {
                int64_t nc = 0;
                for (int64_t i = 0; i < n_inv; ++i)
                    if (out[i].cfg >= 0) nc += c->h_ncfg[c->h_dag_op_off[dag[i]] + op_local[i]];
                snprintf(scored, sizeof scored, "%lld", (long long)nc);
                if (dev_ms > 0.f) snprintf(cps, sizeof cps, "%.6g", (double)nc / (1e-3 * dev_ms));
            }
        }
        fprintf(c->stats,
                "{\"call\": %lld, \"n_inv\": %lld, \"now_us\": %lld, \"method\": \"%s\", \"launches\": %d, "
                "\"graph\": %s, \"invalid\": %llu, \"timeout\": %s, \"device_us\": %.3f, \"host_us\": %.3f, "
                "\"inputs\": \"%s\", \"inv_per_s\": %.6g, \"feasible\": %s, \"configs_scored\": %s, "
                "\"configs_per_s\": %s}\n",
                (long long)c->stats_calls++, (long long)n_inv, (long long)now_us,
                c->method == LLAMA_METHOD_STAIRCASE ? "staircase" : "scan", c->last_launches,
                c->opts.use_graph && !c->tracing ? "true" : "false", c->h_ctrl[0], c->h_ctrl[1] ? "true" : "false",
                1e3 * dev_ms, host_us, rd && ro && rs ? "read in place" : "copied",
                dev_ms > 0.f ? (double)n_inv / (1e-3 * dev_ms) : 0.0, feas, scored, cps);
        fflush(c->stats);
    }
    if (c->h_ctrl[1])
        return c->fail(LLAMA_ETIMEOUT, "schedule: a bounded device wait gave up (bucketing barrier or table "
                                       "staging); valid invocations are flagged LLAMA_FLAG_TIMEOUT in out");
    if (c->h_ctrl[0])
        return c->fail(LLAMA_EINVAL, "schedule: some invocations are invalid (flagged in out)");
    return LLAMA_OK;
}

extern "C" int llama_critical_path(llama_ctx *c, int64_t *cp_us) {
    if (!c) return LLAMA_EINVAL;
    if (!cp_us) return c->fail(LLAMA_EINVAL, "critical_path: null output");
    int rc = check_ready(c);
    if (rc) return rc;
    DeviceGuard g(c->opts.device);
    const DevProblem P = make_problem(c);
    k_critical_path<<<c->n_dags, 64, 0, c->stream>>>(P, c->topo.as<int32_t>(), c->lvl_off.as<int32_t>(),
                                                     c->dag_lvl.as<int32_t>());
    LL_CUDA(c, cudaGetLastError());
    LL_CUDA(c, cudaMemcpyAsync(cp_us, c->cp.p, 8 * (size_t)c->n_ops, cudaMemcpyDeviceToHost, c->stream));
    LL_CUDA(c, cudaStreamSynchronize(c->stream));
    return LLAMA_OK;
}

extern "C" int llama_slack(llama_ctx *c, int64_t n_inv, const int32_t *dag, const int32_t *op_local,
                           const int64_t *start_us, int64_t now_us, int32_t *slack_us) {
    if (!c) return LLAMA_EINVAL;
    int rc = check_inv_args(c, n_inv, dag, op_local, start_us, slack_us);
    if (rc) return rc;
    if ((rc = check_ready(c))) return rc;
    if (n_inv == 0) return LLAMA_OK;
    DeviceGuard g(c->opts.device);
    const int H = c->opts.n_hw;
    const bool dd = is_device_ptr(dag), od = is_device_ptr(op_local), sd = is_device_ptr(start_us),
               outd = is_device_ptr(slack_us);
    if (!(dd && od && sd && outd) && (rc = ensure_stage(c, n_inv))) return rc;
    cudaStream_t s = c->stream;
    const int32_t *d_dag = dd ? dag : c->s_dag.as<int32_t>();
    const int32_t *d_opl = od ? op_local : c->s_opl.as<int32_t>();
    const int64_t *d_start = sd ? start_us : c->s_start.as<int64_t>();
    int32_t *d_out = outd ? slack_us : c->s_slack.as<int32_t>();
    if (!dd) LL_CUDA(c, cudaMemcpyAsync((void *)d_dag, dag, 4 * n_inv, cudaMemcpyHostToDevice, s));
    if (!od) LL_CUDA(c, cudaMemcpyAsync((void *)d_opl, op_local, 4 * n_inv, cudaMemcpyHostToDevice, s));
    if (!sd) LL_CUDA(c, cudaMemcpyAsync((void *)d_start, start_us, 8 * n_inv, cudaMemcpyHostToDevice, s));
    const DevProblem P = make_problem(c);
    k_critical_path<<<c->n_dags, 64, 0, s>>>(P, c->topo.as<int32_t>(), c->lvl_off.as<int32_t>(),
                                             c->dag_lvl.as<int32_t>());
    k_slack<<<grid_for(c, n_inv, 256), 256, 0, s>>>(P, n_inv, d_dag, d_opl, d_start, now_us, d_out);
    LL_CUDA(c, cudaGetLastError());
    if (!outd) LL_CUDA(c, cudaMemcpyAsync(slack_us, d_out, 4 * n_inv * H, cudaMemcpyDeviceToHost, s));
    LL_CUDA(c, cudaStreamSynchronize(s));
    return LLAMA_OK;
}
