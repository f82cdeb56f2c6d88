// kernels.cu -- sm_103a kernels of the scheduling step.
//
//   k_prepare   critical path per op (Alg. 1's RemainingPathLatency maximised over
//               paths; one CTA per DAG, level-synchronous from the sinks upwards),
//               validation and per-op counts of the invocations, and the bucket
//               layout (last CTA).
//   k_scatter   bucket the invocations by operation and compute their slack per
//               backend (Algorithm 1 through the critical path).
//   k_score     Eq. 1 over every configuration of each invocation's operation and
//               the argmin, on the rank-encoded tables.
//   k_encode_*  build the rank encoding of the tables (once per llama_set_profiles).
//
// Rank encoding.  For a configuration x, Eq. 1's value in each branch does not
// depend on the invocation: the feasible branch is C(x)/B(x) and the
// infeasible one is C/B + alpha-term (ALPHA) or "after every feasible
// configuration, by latency" (COST_FIRST, whose infeasible choice is the fixed
// fastest configuration of the op).  Only which branch applies depends on the
// invocation's slack.  So each branch value is replaced by its rank in the
// op's total order of (value, index) pairs: rf(x) for the feasible branch and
// ri(x) for the infeasible one.  Ranks are < 2 * 8192 and fit 16 bits; the
// argmin of ranks is the argmin of (value, index) exactly, ties included.
#include <algorithm>
#include <climits>

#include "llama_internal.cuh"

namespace llama {

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// Per-half unsigned 16-bit minimum.
__device__ __forceinline__ uint32_t vmin_u16x2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// Backend lambda(x) of op-local configuration x: the segment containing it.
__device__ __forceinline__ int backend_of(const int32_t *hw_off_v, int H, int x) {
    int lam = 0;
    while (lam + 1 < H && x >= hw_off_v[lam + 1]) ++lam;
    return lam;
}

// ---------------------------------------------------------------------------
// a1 + a3: prepare (critical path, per-op counts, op-ordered aligned prefix)
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool invocation_valid(const DevProblem &P, int32_t d, int32_t o,
                                                 int64_t s, int64_t now) {
    if (d < 0 || d >= P.n_dags) return false;
    if (o < 0 || o >= P.dag_op_off[d + 1] - P.dag_op_off[d]) return false;
    return s >= 0 && s <= now;
}

// Longest remaining reference-latency path of every op of DAG d, op included
// (Algorithm 1's RemainingPathLatency maximised over the paths through op).
// Levels hold the ops of equal height above the sinks (height 0 first), so
// every successor's value is final before its predecessors read it.  A DAG
// that fits is staged in shared memory first (one round of loads), so each
// level costs a barrier instead of a global-memory round trip.
struct CpSmem {
    int64_t cp[kCpSmemOps];
    int64_t ref[kCpSmemOps];
    int32_t rp[kCpSmemOps + 1];
    int32_t col[kCpSmemEdges];
    int32_t topo[kCpSmemOps];
    int32_t lvl[kCpSmemOps + 1];
};

__device__ void critical_path_of_dag(const DevProblem &P, int d, const int32_t *topo,
                                     const int32_t *lvl_off, const int32_t *dag_lvl, CpSmem &sm) {
    const int lo = P.dag_op_off[d], hi = P.dag_op_off[d + 1], n = hi - lo;
    const int e_lo = P.row_ptr[lo], ne = P.row_ptr[hi] - e_lo;
    const int l_lo = dag_lvl[d], nl = dag_lvl[d + 1] - l_lo;
    if (n <= kCpSmemOps && ne <= kCpSmemEdges) {
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const int v = lo + k;
            sm.ref[k] = (int64_t)P.lat[P.cfg_off[v] + P.ref_cfg[v]];
            sm.rp[k] = P.row_ptr[v] - e_lo;
            sm.topo[k] = topo[v] - lo;
        }
        for (int k = threadIdx.x; k < ne; k += blockDim.x) sm.col[k] = P.col[e_lo + k] - lo;
        for (int k = threadIdx.x; k <= nl; k += blockDim.x) sm.lvl[k] = lvl_off[l_lo + k] - lo;
        if (threadIdx.x == 0) sm.rp[n] = ne;
        __syncthreads();
        for (int l = 0; l < nl; ++l) {
            for (int p = sm.lvl[l] + (int)threadIdx.x; p < sm.lvl[l + 1]; p += blockDim.x) {
                const int v = sm.topo[p];
                int64_t best = 0;
                for (int e = sm.rp[v]; e < sm.rp[v + 1]; ++e) best = max(best, sm.cp[sm.col[e]]);
                sm.cp[v] = sm.ref[v] + best;
            }
            __syncthreads();
        }
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            P.ref[lo + k] = sm.ref[k];
            P.cp[lo + k] = sm.cp[k];
        }
        return;
    }
    for (int v = lo + (int)threadIdx.x; v < hi; v += blockDim.x)
        P.ref[v] = (int64_t)P.lat[P.cfg_off[v] + P.ref_cfg[v]];
    __syncthreads();
    for (int l = dag_lvl[d]; l < dag_lvl[d + 1]; ++l) {
        for (int p = lvl_off[l] + (int)threadIdx.x; p < lvl_off[l + 1]; p += blockDim.x) {
            const int v = topo[p];
            int64_t best = 0;
            for (int e = P.row_ptr[v]; e < P.row_ptr[v + 1]; ++e) best = max(best, P.cp[P.col[e]]);
            P.cp[v] = P.ref[v] + best;
        }
        __syncthreads();
    }
}

__global__ void k_critical_path(DevProblem P, const int32_t *topo, const int32_t *lvl_off,
                                const int32_t *dag_lvl) {
    __shared__ CpSmem sm;
    critical_path_of_dag(P, blockIdx.x, topo, lvl_off, dag_lvl, sm);
}

// Number of lanes (log2) working on one invocation of an op whose padded table
// has nvec 8-configuration vectors: enough that each lane scans about
// min_vpl vectors, at most one CTA.
__device__ __forceinline__ int lanes_log2_for(int32_t nvec, int32_t min_vpl) {
    int lg = 0;
    while (lg < kScoreThreadsLog2 && (nvec >> (lg + 1)) >= min_vpl) ++lg;
    return lg;
}

// Tiles of one op with cnt invocations: full tiles of kScoreThreads >> lg
// invocations at 2^lg lanes each, then one tail tile whose invocations get as
// many lanes as fill a CTA (at most the op's vector count, rounded up).
__device__ __forceinline__ int32_t tiles_of_op(int32_t cnt, int lg) {
    const int32_t per = kScoreThreads >> lg;
    return cnt / per + (cnt % per ? 1 : 0);
}

// Blocks [0, n_dags) compute the critical path of one DAG each; the others
// validate invocations, count them per op (one counter per 128-byte line, so
// concurrent atomics on different ops never share a line) and prefetch the
// encoded tables into L2.  The last block to finish lays out the buckets and
// the scoring tiles, ops in the order P.op_order (largest tables first).
__global__ void __launch_bounds__(256) k_prepare(DevProblem P, int64_t n_inv, const int32_t *dag,
                                                 const int32_t *op_local, const int64_t *start,
                                                 int64_t now, BucketScratch S, llama_decision *out,
                                                 const int32_t *topo, const int32_t *lvl_off,
                                                 const int32_t *dag_lvl, int32_t min_vpl) {
    __shared__ int32_t warp_pos[32], warp_til[32];
    __shared__ int last;
    __shared__ CpSmem sm;
    if ((int)blockIdx.x < P.n_dags) {
        critical_path_of_dag(P, blockIdx.x, topo, lvl_off, dag_lvl, sm);
    } else {
        const int64_t nb = gridDim.x - P.n_dags;
        for (int64_t i = (blockIdx.x - P.n_dags) * (int64_t)blockDim.x + threadIdx.x; i < n_inv;
             i += nb * blockDim.x) {
            const int32_t d = dag[i], o = op_local[i];
            if (!invocation_valid(P, d, o, start[i], now)) {
                S.gop[i] = -1;
                llama_decision bad;
                bad.cfg = -1;
                bad.lat = 0;
                bad.cost = 0;
                bad.slack = 0;
                bad.flags = LLAMA_FLAG_INVALID;
                out[i] = bad;
                atomicAdd(&S.ctrl[kCtrlInvalid], 1ull);
                continue;
            }
            const int32_t g = P.dag_op_off[d] + o;
            S.gop[i] = g;
            S.slot[i] = atomicAdd(&S.cnt[(int64_t)g * kCntStride], 1);
        }
        // Pull the encoded tables into L2 while the buckets are laid out, so the
        // scoring kernel's staging does not wait on DRAM.
        if (P.prefetch_lines > 0) {
            // each array is 2*n_pad bytes; line l < ceil(2*n_pad / 128) starts inside it
            const char *arr[4] = {reinterpret_cast<const char *>(P.lat_lo),
                                  reinterpret_cast<const char *>(P.lat_hi),
                                  reinterpret_cast<const char *>(P.rf),
                                  reinterpret_cast<const char *>(P.df)};
            const int n_arr = P.df ? 4 : 3;
            for (int64_t l = (blockIdx.x - P.n_dags) * (int64_t)blockDim.x + threadIdx.x;
                 l < P.prefetch_lines * n_arr; l += nb * blockDim.x) {
                const char *a = arr[l % n_arr] + 128 * (l / n_arr);
                asm volatile("prefetch.global.L2::evict_last [%0];" ::"l"(a));
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&S.ctrl[kCtrlTicket], 1ull) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();

    // exclusive prefixes, in op_order, of the bucket sizes and of the tile counts
    const int n = P.n_ops, T = blockDim.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int per = (n + T - 1) / T;
    const int b = min(n, tid * per), e = min(n, b + per);
    int32_t c = 0, t = 0;
    for (int k = b; k < e; ++k) {
        const int32_t v = P.op_order[k];
        const int32_t ck = __ldcg(&S.cnt[(int64_t)v * kCntStride]);
        const int32_t nvec = (int32_t)((P.pad_off[v + 1] - P.pad_off[v]) / kVec);
        c += ck;
        t += tiles_of_op(ck, lanes_log2_for(nvec, min_vpl));
    }
    int32_t ci = c, ti = t;
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t uc = __shfl_up_sync(0xffffffffu, ci, o);
        const int32_t ut = __shfl_up_sync(0xffffffffu, ti, o);
        if (lane >= o) { ci += uc; ti += ut; }
    }
    if (lane == 31) { warp_pos[wid] = ci; warp_til[wid] = ti; }
    __syncthreads();
    if (wid == 0) {
        const int nw = T >> 5;
        int32_t wc = lane < nw ? warp_pos[lane] : 0, wt = lane < nw ? warp_til[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t uc = __shfl_up_sync(0xffffffffu, wc, o);
            const int32_t ut = __shfl_up_sync(0xffffffffu, wt, o);
            if (lane >= o) { wc += uc; wt += ut; }
        }
        if (lane < nw) { warp_pos[lane] = wc; warp_til[lane] = wt; }
    }
    __syncthreads();
    int32_t c0 = ci - c + (wid > 0 ? warp_pos[wid - 1] : 0);
    int32_t t0 = ti - t + (wid > 0 ? warp_til[wid - 1] : 0);
    for (int k = b; k < e; ++k) {
        const int32_t v = P.op_order[k];
        const int32_t ck = __ldcg(&S.cnt[(int64_t)v * kCntStride]);
        const int32_t nvec = (int32_t)((P.pad_off[v + 1] - P.pad_off[v]) / kVec);
        const int lg = lanes_log2_for(nvec, min_vpl);
        const int32_t per_tile = kScoreThreads >> lg;
        S.op_start[v] = c0;
        int32_t j = 0;
        for (; j + per_tile <= ck; j += per_tile) S.tiles[t0++] = make_int4(v, j, per_tile, lg);
        if (j < ck) {
            // tail: more lanes per invocation, up to a CTA, no more than the op has vectors
            const int32_t m = ck - j;
            int tlg = lg;
            while (tlg < kScoreThreadsLog2 && (m << (tlg + 1)) <= kScoreThreads && (1 << tlg) < nvec) ++tlg;
            S.tiles[t0++] = make_int4(v, j, m, tlg);
        }
        c0 += ck;
    }
    if (tid == T - 1) {
        S.ctrl[kCtrlPositions] = (unsigned long long)c0;
        S.ctrl[kCtrlTiles] = (unsigned long long)t0;
    }
}

// a2 fused with a3's scatter: place each invocation in its op's bucket and
// compute its slack for every backend (Algorithm 1 through the critical path).
__global__ void __launch_bounds__(256) k_scatter(DevProblem P, int64_t n_inv, const int32_t *dag,
                                                 const int64_t *start, int64_t now, BucketScratch S) {
    // let the scoring kernel start staging its tables while this one runs
    asm volatile("griddepcontrol.launch_dependents;");
    const int H = P.n_hw;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_inv;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = S.gop[i];
        if (g < 0) continue;
        S.b_inv[S.op_start[g] + S.slot[i]] = (int32_t)i;
        const int64_t r_base = P.slo[dag[i]] - (now - start[i]);
        const int64_t ref = P.ref[g], cp = P.cp[g];
        for (int h = 0; h < H; ++h) S.b_slack[i * H + h] = slack_of(ref, cp, r_base - P.q[h]);
    }
}

// Slack of every invocation for every backend, without bucketing.
__global__ void k_slack(DevProblem P, int64_t n_inv, const int32_t *dag, const int32_t *op_local,
                        const int64_t *start, int64_t now, int32_t *slack_out) {
    const int H = P.n_hw;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_inv;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = dag[i], o = op_local[i];
        if (!invocation_valid(P, d, o, start[i], now)) {
            for (int h = 0; h < H; ++h) slack_out[i * H + h] = -1;
            continue;
        }
        const int32_t g = P.dag_op_off[d] + o;
        const int64_t r_base = P.slo[d] - (now - start[i]);
        for (int h = 0; h < H; ++h) slack_out[i * H + h] = slack_of(P.ref[g], P.cp[g], r_base - P.q[h]);
    }
}

// ---------------------------------------------------------------------------
// a4: scoring
// ---------------------------------------------------------------------------

// Eight configurations against slack-1 = sm1: t = sm1 - L is negative exactly
// when L >= slack (infeasible).  Cost-first: the sign bits of two configs are
// moved to bits 15 and 31 and OR-ed onto their feasible-branch ranks (an
// infeasible key is >= 0x8000, above every feasible one); alpha: the sign
// bytes are replicated into a 0xFFFF mask that selects the infeasible-branch
// rank rf ^ df.  Then a per-half unsigned 16-bit running minimum.
__device__ __forceinline__ uint32_t scan8_cost_first(uint32_t best, int32_t sm1, int4 l0, int4 l1,
                                                     uint4 rk) {
    best = vmin_u16x2(best, rk.x | (prmt(sm1 - l0.x, sm1 - l0.y, 0x7430u) & 0x80008000u));
    best = vmin_u16x2(best, rk.y | (prmt(sm1 - l0.z, sm1 - l0.w, 0x7430u) & 0x80008000u));
    best = vmin_u16x2(best, rk.z | (prmt(sm1 - l1.x, sm1 - l1.y, 0x7430u) & 0x80008000u));
    best = vmin_u16x2(best, rk.w | (prmt(sm1 - l1.z, sm1 - l1.w, 0x7430u) & 0x80008000u));
    return best;
}

__device__ __forceinline__ uint32_t scan8_alpha(uint32_t best, int32_t sm1, int4 l0, int4 l1,
                                                uint4 rk, uint4 dk) {
    best = vmin_u16x2(best, rk.x ^ (dk.x & prmt(sm1 - l0.x, sm1 - l0.y, 0xFFBBu)));
    best = vmin_u16x2(best, rk.y ^ (dk.y & prmt(sm1 - l0.z, sm1 - l0.w, 0xFFBBu)));
    best = vmin_u16x2(best, rk.z ^ (dk.z & prmt(sm1 - l1.x, sm1 - l1.y, 0xFFBBu)));
    best = vmin_u16x2(best, rk.w ^ (dk.w & prmt(sm1 - l1.z, sm1 - l1.w, 0xFFBBu)));
    return best;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Wait until the mbarrier completes the phase with the given parity, for a
// bounded number of attempts.  Returns false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (int it = 0; it < kMaxWaitTries; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

// One bulk copy global -> shared, completing on the mbarrier (16-byte aligned
// addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
        ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// Persistent CTAs walk the tile list (op, first invocation j0, m invocations,
// 2^lg lanes each).  For a tile, the op's encoded table is staged into shared
// memory by TMA bulk copies, in chunks of at most `chunk` entries (a multiple
// of 8); each group of 2^lg lanes scores one invocation: lane s takes the
// vectors q = s mod 2^lg of every backend segment, against that segment's
// slack.  Groups reduce with shuffles (and through shared memory when a group
// spans several warps); lane 0 decodes the winning rank.
template <int MODE>
__device__ __forceinline__ void score_body(const DevProblem &P, const BucketScratch &S,
                                           llama_decision *out, int32_t chunk) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // chunk entries: latency planes (entries 0-3 and 4-7 of each vector), ranks
    int32_t *lo_s = reinterpret_cast<int32_t *>(smem_raw);
    int32_t *hi_s = lo_s + chunk / 2;
    uint16_t *rf_s = reinterpret_cast<uint16_t *>(hi_s + chunk / 2);
    uint16_t *df_s = rf_s + chunk;
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ uint32_t red[kScoreThreads / 32];
    const int tid = threadIdx.x, H = P.n_hw;
    const uint32_t bar = smem_addr(&mbar);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t phase = 0;
    bool ok = true;
    // tiles and buckets come from k_prepare (complete before k_scatter began);
    // b_inv and b_slack come from k_scatter: wait for it before the first read
    const int64_t n_tiles = (int64_t)S.ctrl[kCtrlTiles];
    bool scatter_done = false;
    for (int64_t ti = blockIdx.x; ti < n_tiles && ok; ti += gridDim.x) {
        const int4 tile = S.tiles[ti];
        const int32_t v = tile.x, j0 = tile.y, m = tile.z, lg = tile.w;
        const int L = 1 << lg;
        const bool active = tid < (m << lg);
        const int g = tid >> lg, s = tid & (L - 1);
        const int64_t p0 = P.pad_off[v];
        const int32_t npad = (int32_t)(P.pad_off[v + 1] - p0);
        const int32_t *sp = P.seg_pad + (int64_t)v * (H + 1);
        if (!scatter_done) {
            asm volatile("griddepcontrol.wait;" ::: "memory");
            scatter_done = true;
        }
        int32_t i = -1;
        if (active) i = S.b_inv[S.op_start[v] + j0 + g];
        const int32_t *slk = S.b_slack + (int64_t)(i < 0 ? 0 : i) * H;
        uint32_t best = 0xFFFFFFFFu;
        for (int32_t c0 = 0; c0 < npad; c0 += chunk) {
            const int32_t cn = min(chunk, npad - c0);
            __syncthreads();  // every thread is done with the previous chunk or tile
            if (tid == 0) {
                // the generic-proxy reads of the previous chunk are complete (barrier
                // above); order them before the async-proxy writes that follow
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                const uint32_t bytes = (uint32_t)cn * (MODE == LLAMA_MODE_ALPHA ? 8u : 6u);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                             ::"r"(bar), "r"(bytes) : "memory");
                bulk_g2s(lo_s, P.lat_lo + (p0 + c0) / 2, 2u * cn, bar);
                bulk_g2s(hi_s, P.lat_hi + (p0 + c0) / 2, 2u * cn, bar);
                bulk_g2s(rf_s, P.rf + p0 + c0, 2u * cn, bar);
                if (MODE == LLAMA_MODE_ALPHA) bulk_g2s(df_s, P.df + p0 + c0, 2u * cn, bar);
            }
            // every thread must agree before any leaves the barrier sequence
            if (!__syncthreads_and(mbar_wait(bar, phase))) {
                ok = false;
                break;
            }
            phase ^= 1u;
            if (active) {
                const int qc0 = c0 / kVec, qc1 = (c0 + cn) / kVec;
                const int4 *lo4 = reinterpret_cast<const int4 *>(lo_s);
                const int4 *hi4 = reinterpret_cast<const int4 *>(hi_s);
                const uint4 *rf4 = reinterpret_cast<const uint4 *>(rf_s);
                const uint4 *df4 = reinterpret_cast<const uint4 *>(df_s);
                for (int h = 0; h < H; ++h) {
                    const int a = max(__ldg(sp + h) / kVec, qc0), b = min(__ldg(sp + h + 1) / kVec, qc1);
                    if (a >= b) continue;
                    const int32_t sm1 = slk[h] - 1;
                    for (int q = a + ((s - a) & (L - 1)); q < b; q += L) {
                        const int r = q - qc0;
                        if (MODE == LLAMA_MODE_ALPHA)
                            best = scan8_alpha(best, sm1, lo4[r], hi4[r], rf4[r], df4[r]);
                        else
                            best = scan8_cost_first(best, sm1, lo4[r], hi4[r], rf4[r]);
                    }
                }
            }
        }
        if (!ok) break;
        uint32_t key = active ? min(best & 0xFFFFu, best >> 16) : 0xFFFFu;
        const int wl = L < 32 ? L : 32;
        for (int o = 1; o < wl; o <<= 1) key = min(key, __shfl_xor_sync(0xffffffffu, key, o));
        if (L > 32) {
            // a group spans L/32 warps: combine the warps' minima in shared memory
            if ((tid & 31) == 0) red[tid >> 5] = key;
            __syncthreads();
            if (s == 0) {
                for (int w = 1; w < (L >> 5); ++w) key = min(key, red[(tid >> 5) + w]);
            }
        }
        if (active && s == 0) {
            const int64_t c_base = P.cfg_off[v];
            int32_t idx;
            if (MODE == LLAMA_MODE_ALPHA) idx = P.inv[2 * c_base + key];
            else idx = key < 0x8000u ? (int32_t)P.inv[2 * c_base + key] : P.fast[v];
            const int64_t gx = c_base + idx;
            const int32_t Lx = P.lat[gx];
            const int lam = backend_of(P.hw_off + (int64_t)v * (H + 1), H, idx);
            const int32_t sl = S.b_slack[(int64_t)i * H + lam];
            llama_decision dsn;
            dsn.cfg = idx;
            dsn.lat = Lx;
            dsn.cost = P.cost[gx];
            dsn.slack = sl;
            dsn.flags = Lx < sl ? LLAMA_FLAG_FEASIBLE : 0;
            out[i] = dsn;
        }
    }
    if (!ok) {
        // a staging copy never completed: report it, wait (bounded) for the copy
        // to land so no transfer targets this CTA's shared memory after exit
        if (tid == 0) atomicOr(&S.ctrl[kCtrlTimeout], 1ull);
        mbar_wait(bar, phase);
    }
}

__global__ void __launch_bounds__(kScoreThreads)
    k_score_cost_first(DevProblem P, BucketScratch S, llama_decision *out, int32_t chunk) {
    score_body<LLAMA_MODE_COST_FIRST>(P, S, out, chunk);
}

__global__ void __launch_bounds__(kScoreThreads)
    k_score_alpha(DevProblem P, BucketScratch S, llama_decision *out, int32_t chunk) {
    score_body<LLAMA_MODE_ALPHA>(P, S, out, chunk);
}

// ---------------------------------------------------------------------------
// The launch sequence of one scheduling call
// ---------------------------------------------------------------------------

int64_t max_tiles(int64_t n_inv, int32_t n_ops) { return n_inv + n_ops; }

cudaError_t enqueue_schedule(const ContextView &v, const BucketScratch &S, int64_t n_inv,
                             const int32_t *dag, const int32_t *op_local, const int64_t *start,
                             int64_t now, llama_decision *out, cudaStream_t s,
                             const cudaEvent_t *trace) {
    // external: when captured into a graph the records become event-record nodes
    auto mark = [&](int k) { if (trace) cudaEventRecordWithFlags(trace[k], s, cudaEventRecordExternal); };
    mark(0);
    cudaError_t e = cudaMemsetAsync(S.cnt, 0, sizeof(int32_t) * kCntStride * (size_t)v.n_ops, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(S.ctrl, 0, sizeof(unsigned long long) * kCtrlWords, s);
    if (e != cudaSuccess) return e;
    const int count_blocks =
        (int)std::max<int64_t>(1, std::min<int64_t>((n_inv + 255) / 256, (int64_t)v.num_sms * 8));
    k_prepare<<<v.n_dags + count_blocks, 256, 0, s>>>(v.P, n_inv, dag, op_local, start, now, S, out,
                                                      v.topo, v.lvl_off, v.dag_lvl, v.min_vpl);
    mark(1);
    const int gi = (int)std::max<int64_t>(1, std::min<int64_t>((n_inv + 255) / 256, (int64_t)v.num_sms * 16));
    k_scatter<<<gi, 256, 0, s>>>(v.P, n_inv, dag, start, now, S);
    mark(2);
    // the scoring kernel may launch before k_scatter completes (it waits on
    // griddepcontrol.wait before reading k_scatter's output)
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(v.score_grid);
    cfg.blockDim = dim3(kScoreThreads);
    cfg.dynamicSmemBytes = v.score_smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = trace ? 0 : 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (v.mode == LLAMA_MODE_ALPHA)
        e = cudaLaunchKernelEx(&cfg, k_score_alpha, v.P, S, out, v.score_chunk);
    else
        e = cudaLaunchKernelEx(&cfg, k_score_cost_first, v.P, S, out, v.score_chunk);
    if (e != cudaSuccess) return e;
    mark(3);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Encoding of the tables (llama_set_profiles)
// ---------------------------------------------------------------------------

// One CTA per op: latencies into the padded layout (INT32_MAX at pads, which no
// slack can exceed), ranks initialised to the pad rank, and the op's fastest
// configuration argmin (L, index).
__global__ void k_encode_pad(DevProblem P, int32_t *lat_lo, int32_t *lat_hi, uint16_t *rf,
                             uint16_t *df, int32_t *fast) {
    __shared__ int64_t red[32];
    const int v = blockIdx.x, H = P.n_hw;
    const int64_t c0 = P.cfg_off[v], p0 = P.pad_off[v];
    const int32_t *hw = P.hw_off + (int64_t)v * (H + 1);
    const int32_t *sp = P.seg_pad + (int64_t)v * (H + 1);
    for (int h = 0; h < H; ++h) {
        const int src_n = hw[h + 1] - hw[h], dst_n = sp[h + 1] - sp[h];
        for (int k = threadIdx.x; k < dst_n; k += blockDim.x) {
            const int64_t dst = p0 + sp[h] + k;  // padded position; vector dst/8, entry dst%8
            const int32_t L = k < src_n ? P.lat[c0 + hw[h] + k] : INT32_MAX;
            const int64_t plane = dst / kVec * 4 + dst % 4;
            if (dst % kVec < 4) lat_lo[plane] = L; else lat_hi[plane] = L;
            rf[dst] = kPadRank;
            if (df) df[dst] = 0;
        }
    }
    // argmin over (L, index): pack L (31 bits) above the index (13 bits)
    const int n = (int)(P.cfg_off[v + 1] - c0);
    int64_t best = LLONG_MAX;
    for (int x = threadIdx.x; x < n; x += blockDim.x)
        best = min(best, ((int64_t)P.lat[c0 + x] << 16) | x);
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x < 32) {
        best = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : LLONG_MAX;
        for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
        if (threadIdx.x == 0) fast[v] = (int32_t)(best & 0xFFFF);
    }
}

// Eq. 1's infeasible branch in unsigned 64-bit: alpha_num*L*R < 2^63 and
// alpha_den*B*R_total < 2^63 by the validated bounds; the sum saturates.
__device__ __forceinline__ uint64_t alpha_infeasible_objective(const DevProblem &P, int64_t g, int h) {
    const uint64_t num = (uint64_t)P.alpha_num * (uint64_t)P.lat[g] * (uint64_t)P.res[g];
    const uint64_t den = (uint64_t)P.alpha_den * (uint64_t)P.batch[g] * (uint64_t)P.res_total[h];
    const uint64_t obj = (uint64_t)P.cost[g] + num / den;
    return obj > (uint64_t)LLONG_MAX ? (uint64_t)LLONG_MAX : obj;
}

// One CTA per op: sort the op's (objective, tag) pairs in shared memory with a
// bitonic network and write the ranks.  COST_FIRST sorts (C/B, x); ALPHA sorts
// the 2n values {(C/B, 2x), (infeasible objective, 2x+1)} jointly.
__global__ void k_encode_rank(DevProblem P, int32_t sort_cap, uint16_t *rf, uint16_t *df,
                              uint16_t *inv) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *key = reinterpret_cast<uint64_t *>(smem_raw);
    uint32_t *tag = reinterpret_cast<uint32_t *>(smem_raw + 8 * (size_t)sort_cap);
    const int v = blockIdx.x, H = P.n_hw, T = blockDim.x;
    const bool alpha = P.mode == LLAMA_MODE_ALPHA;
    const int64_t c0 = P.cfg_off[v], p0 = P.pad_off[v];
    const int n = (int)(P.cfg_off[v + 1] - c0);
    const int cnt = alpha ? 2 * n : n;
    int N = 1;
    while (N < cnt) N <<= 1;
    const int32_t *hw = P.hw_off + (int64_t)v * (H + 1);
    const int32_t *sp = P.seg_pad + (int64_t)v * (H + 1);

    for (int k = threadIdx.x; k < N; k += T) {
        if (k < cnt) {
            const int x = alpha ? (k >> 1) : k;
            if (alpha && (k & 1)) key[k] = alpha_infeasible_objective(P, c0 + x, backend_of(hw, H, x));
            else key[k] = (uint64_t)P.cost[c0 + x];
            tag[k] = (uint32_t)k;
        } else {
            key[k] = ~0ull;
            tag[k] = ~0u;
        }
    }
    __syncthreads();
    for (int k = 2; k <= N; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < N; i += T) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    const bool gt = key[i] > key[ixj] || (key[i] == key[ixj] && tag[i] > tag[ixj]);
                    if (gt == up) {
                        const uint64_t tk = key[i]; key[i] = key[ixj]; key[ixj] = tk;
                        const uint32_t tt = tag[i]; tag[i] = tag[ixj]; tag[ixj] = tt;
                    }
                }
            }
            __syncthreads();
        }
    }
    // ranks -> padded positions; for ALPHA collect rf/ri per x first (reusing key[])
    uint16_t *rf_tmp = reinterpret_cast<uint16_t *>(key);
    uint16_t *ri_tmp = rf_tmp + n;
    for (int r = threadIdx.x; r < cnt; r += T) {
        const uint32_t t = tag[r];
        const int x = alpha ? (int)(t >> 1) : (int)t;
        inv[2 * c0 + r] = (uint16_t)x;
        if (alpha) {
            if (t & 1) ri_tmp[x] = (uint16_t)r; else rf_tmp[x] = (uint16_t)r;
        } else {
            const int lam = backend_of(hw, H, x);
            rf[p0 + sp[lam] + (x - hw[lam])] = (uint16_t)r;
        }
    }
    if (!alpha) return;
    __syncthreads();
    for (int x = threadIdx.x; x < n; x += T) {
        const int lam = backend_of(hw, H, x);
        const int64_t dst = p0 + sp[lam] + (x - hw[lam]);
        rf[dst] = rf_tmp[x];
        df[dst] = (uint16_t)(rf_tmp[x] ^ ri_tmp[x]);
    }
}

}  // namespace llama
