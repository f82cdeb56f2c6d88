// kernels.cu -- sm_103a kernels of the scheduling step.
//
//   k_bucket    one cooperative launch: critical path per op (Alg. 1's
//               RemainingPathLatency maximised over paths; one CTA per DAG,
//               level-synchronous from the sinks upwards), validation and per-op
//               counts of the invocations, bucket and tile layout; grid barrier;
//               then the invocations are placed in their op's bucket and their
//               slack per backend computed (Algorithm 1 through the critical path).
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

// Whether a decode key indexes op v's decode table: below twice its
// configurations (alpha: the joint ranks), below its configurations for a
// feasible-branch rank (cost-first; 0x8000 and above decode the fastest
// configuration).  Evaluated in the -DLLAMA_CHECK build only.
__device__ __forceinline__ bool decode_key_ok(const DevProblem &P, int32_t v, uint32_t key, int mode) {
#ifdef LLAMA_CHECK
    if (v < 0 || v >= P.n_ops) return false;
    const int64_t n = P.cfg_off[v + 1] - P.cfg_off[v];
    return mode == LLAMA_MODE_ALPHA ? (int64_t)key < 2 * n : (key >= 0x8000u || (int64_t)key < n);
#else
    return true;
#endif
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

// invocation_valid from the DAG's record (one 16-byte load: op range and SLO);
// for a valid invocation also its global op g and its remaining time before
// queueing, rbase = SLO - elapsed (Algorithm 1).
__device__ __forceinline__ bool invocation_op(const DevProblem &P, int32_t d, int32_t o, int64_t s, int64_t now,
                                              int32_t &g, int64_t &rbase) {
    if (d < 0 || d >= P.n_dags) return false;
    const int4 di = __ldg(P.dag_info + d);
    if (o < 0 || o >= di.y - di.x || s < 0 || s > now) return false;
    g = di.x + o;
    rbase = (int64_t)(((uint64_t)(uint32_t)di.w << 32) | (uint32_t)di.z) - (now - s);
    return true;
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
    int32_t pk[kCpPackWords];
};

__device__ void critical_path_of_dag(const DevProblem &P, int d, const int32_t *topo,
                                     const int32_t *lvl_off, const int32_t *dag_lvl, CpSmem &sm) {
    const int64_t off = P.dag_pack_off[d];
    const int nw = (int)(P.dag_pack_off[d + 1] - off);
    if (nw > 0) {
        // the DAG's packed structure in one round of loads: header {first op, ops,
        // edges, levels}, reference-configuration indices, local successor CSR,
        // ops by height, level offsets
        for (int k = threadIdx.x; k < nw; k += blockDim.x) sm.pk[k] = P.dag_pack[off + k];
        __syncthreads();
        const int lo = sm.pk[0], n = sm.pk[1], ne = sm.pk[2], nl = sm.pk[3];
        const int32_t *gidx = sm.pk + 4, *rp = gidx + n, *col = rp + n + 1, *ord = col + ne, *lvl = ord + n;
        for (int k = threadIdx.x; k < n; k += blockDim.x) sm.ref[k] = (int64_t)P.lat[gidx[k]];
        __syncthreads();
        for (int l = 0; l < nl; ++l) {
            for (int p = lvl[l] + (int)threadIdx.x; p < lvl[l + 1]; p += blockDim.x) {
                const int v = ord[p];
                int64_t best = 0;
                for (int e = rp[v]; e < rp[v + 1]; ++e) best = max(best, sm.cp[col[e]]);
                sm.cp[v] = sm.ref[v] + best;
            }
            __syncthreads();
        }
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            P.ref[lo + k] = sm.ref[k];
            P.cp[lo + k] = sm.cp[k];
            P.cp_magic[lo + k] = ~0ull / (uint64_t)sm.cp[k];
        }
        return;
    }
    // a DAG too large for shared memory: the same levels through global memory
    const int lo = P.dag_op_off[d], hi = P.dag_op_off[d + 1];
    for (int v = lo + (int)threadIdx.x; v < hi; v += blockDim.x)
        P.ref[v] = (int64_t)P.lat[P.ref_gidx[v]];
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
    for (int v = lo + (int)threadIdx.x; v < hi; v += blockDim.x) P.cp_magic[v] = ~0ull / (uint64_t)P.cp[v];
}

// The same levels for a DAG whose packed structure has at most kCpWarpWords
// words (hence at most kCpWarpOps ops), by one warp in its own slice of shared
// memory: a level costs a warp barrier.
struct CpWarpSmem {
    int64_t cp[kCpWarpOps];
    int64_t ref[kCpWarpOps];
    int32_t pk[kCpWarpWords];
};
static_assert(sizeof(CpWarpSmem) * (256 / 32) <= sizeof(CpSmem), "warp slices exceed the block's area");

__device__ void critical_path_of_dag_warp(const DevProblem &P, int64_t off, int nw, CpWarpSmem &w) {
    const int lane = threadIdx.x & 31;
    for (int k = lane; k < nw; k += 32) w.pk[k] = P.dag_pack[off + k];
    __syncwarp();
    const int lo = w.pk[0], n = w.pk[1], ne = w.pk[2], nl = w.pk[3];
    const int32_t *gidx = w.pk + 4, *rp = gidx + n, *col = rp + n + 1, *ord = col + ne, *lvl = ord + n;
    for (int k = lane; k < n; k += 32) w.ref[k] = (int64_t)P.lat[gidx[k]];
    __syncwarp();
    for (int l = 0; l < nl; ++l) {
        for (int p = lvl[l] + lane; p < lvl[l + 1]; p += 32) {
            const int v = ord[p];
            int64_t best = 0;
            for (int e = rp[v]; e < rp[v + 1]; ++e) best = max(best, w.cp[col[e]]);
            w.cp[v] = w.ref[v] + best;
        }
        __syncwarp();
    }
    for (int k = lane; k < n; k += 32) {
        P.ref[lo + k] = w.ref[k];
        P.cp[lo + k] = w.cp[k];
        P.cp_magic[lo + k] = ~0ull / (uint64_t)w.cp[k];
    }
    __syncwarp();  // the slice is reused by the warp's next DAG
}

// Critical paths of the DAGs that block b of nblk takes: small DAGs one per
// warp (DAG b*8 + warp, then strides of nblk*8), then the others one per block
// (DAGs b, b + nblk, ... that did not fit a warp's slice).
__device__ void critical_paths_of_block(const DevProblem &P, int b, int nblk, const int32_t *topo,
                                        const int32_t *lvl_off, const int32_t *dag_lvl, CpSmem &sm) {
    const int nwarp = blockDim.x >> 5, wid = threadIdx.x >> 5;
    CpWarpSmem &ws = reinterpret_cast<CpWarpSmem *>(&sm)[wid];
    for (int d = b * nwarp + wid; d < P.n_dags; d += nblk * nwarp) {
        const int64_t off = P.dag_pack_off[d];
        const int nw = (int)(P.dag_pack_off[d + 1] - off);
        if (nw > 0 && nw <= kCpWarpWords) critical_path_of_dag_warp(P, off, nw, ws);
    }
    __syncthreads();
    for (int d = b; d < P.n_dags; d += nblk) {
        const int nw = (int)(P.dag_pack_off[d + 1] - P.dag_pack_off[d]);
        if (nw > 0 && nw <= kCpWarpWords) continue;
        critical_path_of_dag(P, d, topo, lvl_off, dag_lvl, sm);
        __syncthreads();  // the shared staging area is reused by the next DAG
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

// Tiles of an op with cnt invocations: full tiles of (kScoreThreads >> lg) groups
// of ipt invocations each, then at most one tail tile.  The tail spreads its m
// invocations over more lanes: as many as still fit one CTA, and no more than
// the op has vectors.
__device__ __forceinline__ int32_t full_tiles(int32_t cnt, int lg, int ipt) {
    return cnt / ((kScoreThreads >> lg) * ipt);
}

__device__ __forceinline__ int tail_lanes_log2(int32_t m, int lg, int ipt, int32_t nvec) {
    const int32_t groups = (m + ipt - 1) / ipt;
    while (lg < kScoreThreadsLog2 && (groups << (lg + 1)) <= kScoreThreads && (1 << lg) < nvec) ++lg;
    return lg;
}

// The warp tiles of op v (ck invocations from bucket position pos, tile
// descriptor tx) at tile indices tt, tt + 1, ...: 32 * ipt invocations each
// (lane l of the scoring warp takes its ipt consecutive ones), the last one
// the rest.  Returns the next tile index.
__device__ __forceinline__ int32_t write_warp_tiles(const BucketScratch &S, int32_t v, int32_t pos, int32_t ck,
                                                    int32_t ipt, const int4 &tx, int32_t tt) {
    for (int32_t j = 0; j < ck; j += 32 * ipt, ++tt) {
        S.tiles[2 * tt] = make_int4(v, pos + j, min(32 * ipt, ck - j), 0);
        S.tiles[2 * tt + 1] = tx;
    }
    return tt;
}

// Bucket and tile layout once the counts are final, spread over the counting
// blocks.  Block b of nb owns a contiguous run of ops in the order P.op_order
// (largest tables first); each thread a contiguous run of those.  Positions are
// exclusive prefixes, in that order, of the bucket sizes, of the full tiles and
// of the tail tiles; every op's full tiles come first in the tile list, the
// tails after them.  The warp tiles of the ops from P.n_cta_ops on count as
// tails, so they end the list; the thread that lays out op P.n_cta_ops
// publishes where they start (kCtrlCtaTiles).
struct LayoutRun {
    int32_t kb, ke;          // this thread's ops: op_order[kb .. ke)
    int4 ki[kKeepOps];       // the first kKeepOps of them stay in registers
    int32_t kc[kKeepOps];
    int32_t loc[3];          // bucket positions, full tiles, tail tiles of the run
    int32_t excl[3];         // their exclusive prefixes inside the block
};

// The tiles of an op (bucket-order position k) with ck invocations: full and
// tail tiles of whole CTAs, or, from position P.n_cta_ops on, warp tiles of
// 32 * ipt invocations (counted with the tails: they end the tile list).
__device__ __forceinline__ void op_tiles(int32_t ck, int32_t nvec, int32_t min_vpl, int32_t ipt, bool warp,
                                         int32_t &full, int32_t &tail) {
    if (warp) {
        full = 0;
        tail = (ck + 32 * ipt - 1) / (32 * ipt);
        return;
    }
    const int lg = lanes_log2_for(nvec, min_vpl);
    full = full_tiles(ck, lg, ipt);
    tail = ck > full * ((kScoreThreads >> lg) * ipt) ? 1 : 0;
}

// Inclusive block-wide sums of three values; returns the exclusive prefixes in
// excl[] and the block totals in tot[].
__device__ __forceinline__ void block_scan3(const int32_t loc[3], int32_t excl[3], int32_t tot[3],
                                            int32_t (*warp_sum)[32]) {
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int32_t inc[3] = {loc[0], loc[1], loc[2]};
    for (int o = 1; o < 32; o <<= 1) {
        for (int a = 0; a < 3; ++a) {
            const int32_t u = __shfl_up_sync(0xffffffffu, inc[a], o);
            if (lane >= o) inc[a] += u;
        }
    }
    if (lane == 31)
        for (int a = 0; a < 3; ++a) warp_sum[a][wid] = inc[a];
    __syncthreads();
    if (wid == 0) {
        const int nw = T >> 5;
        for (int a = 0; a < 3; ++a) {
            int32_t w = lane < nw ? warp_sum[a][lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t u = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += u;
            }
            if (lane < nw) warp_sum[a][lane] = w;
        }
    }
    __syncthreads();
    for (int a = 0; a < 3; ++a) {
        excl[a] = inc[a] - loc[a] + (wid > 0 ? warp_sum[a][wid - 1] : 0);
        tot[a] = warp_sum[a][(T >> 5) - 1];
    }
    __syncthreads();  // warp_sum is reused by the caller
}

// Phase 1: this block's ops, summed; the block's totals go to S.blk[b].
__device__ void layout_sums(const DevProblem &P, const BucketScratch &S, int32_t b, int32_t nb,
                            int32_t min_vpl, int32_t ipt, LayoutRun &R, int32_t (*warp_sum)[32]) {
    const int n = P.n_ops, T = blockDim.x, tid = threadIdx.x;
    const int32_t per_blk = (n + nb - 1) / nb;
    const int32_t k0 = min(n, b * per_blk), k1 = min(n, k0 + per_blk);
    const int32_t per = (k1 - k0 + T - 1) / T;
    R.kb = min(k1, k0 + tid * per);
    R.ke = min(k1, R.kb + per);
    R.loc[0] = R.loc[1] = R.loc[2] = 0;
#pragma unroll
    for (int j = 0; j < kKeepOps; ++j)
        if (R.kb + j < R.ke) R.ki[j] = P.ord_info[R.kb + j];
#pragma unroll
    for (int j = 0; j < kKeepOps; ++j)
        if (R.kb + j < R.ke) R.kc[j] = __ldcg(&S.cnt[(int64_t)R.ki[j].x * kCntStride]);
#pragma unroll
    for (int j = 0; j < kKeepOps; ++j) {
        if (R.kb + j >= R.ke) break;
        int32_t f, t;
        op_tiles(R.kc[j], R.ki[j].y, min_vpl, ipt, R.kb + j >= P.n_cta_ops, f, t);
        R.loc[0] += R.kc[j];
        R.loc[1] += f;
        R.loc[2] += t;
    }
    for (int k = R.kb + kKeepOps; k < R.ke; ++k) {
        const int4 oi = P.ord_info[k];
        const int32_t ck = __ldcg(&S.cnt[(int64_t)oi.x * kCntStride]);
        int32_t f, t;
        op_tiles(ck, oi.y, min_vpl, ipt, k >= P.n_cta_ops, f, t);
        R.loc[0] += ck;
        R.loc[1] += f;
        R.loc[2] += t;
    }
    int32_t tot[3];
    block_scan3(R.loc, R.excl, tot, warp_sum);
    if (tid == 0) S.blk[b] = make_int4(tot[0], tot[1], tot[2], 0);
}

// Phase 2 (after every counting block's sums are visible): offsets of this
// block from the sums of the blocks before it, then the buckets and tiles.
__device__ void layout_write(const DevProblem &P, const BucketScratch &S, int32_t b, int32_t nb,
                             int32_t min_vpl, int32_t ipt, const LayoutRun &R, int32_t (*warp_sum)[32]) {
    const int T = blockDim.x, tid = threadIdx.x;
    // before[0..2]: sums of blocks < b; before[3]: full tiles of all blocks
    int32_t acc[4] = {0, 0, 0, 0};
    for (int k = tid; k < nb; k += T) {
        const int4 t = __ldcg(&S.blk[k]);
        if (k < b) acc[0] += t.x, acc[1] += t.y, acc[2] += t.z;
        acc[3] += t.y;
    }
    for (int a = 0; a < 4; ++a)
        for (int o = 16; o > 0; o >>= 1) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], o);
    __shared__ int32_t red[4][32];
    if ((tid & 31) == 0)
        for (int a = 0; a < 4; ++a) red[a][tid >> 5] = acc[a];
    __syncthreads();
    int32_t before[4] = {0, 0, 0, 0};
    for (int w = 0; w < (T >> 5); ++w)
        for (int a = 0; a < 4; ++a) before[a] += red[a][w];
    int32_t pos = before[0] + R.excl[0];
    int32_t tf = before[1] + R.excl[1];
    int32_t tt = before[3] + before[2] + R.excl[2];
    for (int k = R.kb; k < R.ke; ++k) {
        int4 oi;
        int32_t ck;
        if (k - R.kb < kKeepOps) {
            // registers, selected without a runtime index
            oi = R.ki[0], ck = R.kc[0];
#pragma unroll
            for (int j = 1; j < kKeepOps; ++j)
                if (k - R.kb == j) oi = R.ki[j], ck = R.kc[j];
        } else {
            oi = P.ord_info[k];
            ck = __ldcg(&S.cnt[(int64_t)oi.x * kCntStride]);
        }
        const int32_t v = oi.x, nvec = oi.y;
        // {padded entries, distinct latencies, padded offset, first configuration}
        const int4 tx = make_int4(nvec * kVec, oi.w, oi.z, __ldg(P.ord_cbase + k));
        S.op_start[v] = pos;
        if (k >= P.n_cta_ops) {
            if (k == P.n_cta_ops) S.ctrl[kCtrlCtaTiles] = (unsigned long long)tt;
            tt = write_warp_tiles(S, v, pos, ck, ipt, tx, tt);
            pos += ck;
            continue;
        }
        const int lg = lanes_log2_for(nvec, min_vpl);
        const int32_t per_tile = (kScoreThreads >> lg) * ipt;
        int32_t j = 0;
        for (; j + per_tile <= ck; j += per_tile, ++tf) {
            S.tiles[2 * tf] = make_int4(v, pos + j, per_tile, lg);
            S.tiles[2 * tf + 1] = tx;
        }
        if (j < ck) {
            S.tiles[2 * tt] = make_int4(v, pos + j, ck - j, tail_lanes_log2(ck - j, lg, ipt, nvec));
            S.tiles[2 * tt + 1] = tx;
            ++tt;
        }
        pos += ck;
    }
    if (b == nb - 1 && tid == T - 1) {
        // the last thread of the last block ends both prefixes
        S.ctrl[kCtrlPositions] = (unsigned long long)pos;
        S.ctrl[kCtrlTiles] = (unsigned long long)tt;
    }
}

// Bucket layout with no barrier of its own, for profiles whose bucket starts
// fit a block's shared memory: every counting block computes the whole prefix
// over the final counts (ops in bucket order) into op_start_s (by op), and
// block cb of nc writes the tiles of the ops at bucket-order positions
// [cb*tper, (cb+1)*tper).  Positions and tile indices are those of
// layout_sums/layout_write (every op's full tiles first, then the tails).
// Block 0 publishes the numbers of bucket positions and tiles.
__device__ void layout_whole(const DevProblem &P, const BucketScratch &S, int32_t cb, int32_t nc,
                             int32_t min_vpl, int32_t ipt, int32_t *op_start_s, int32_t (*warp_sum)[32]) {
    constexpr int kW = kLayoutWholeOps / 256;  // ops per thread at most (blockDim.x == 256)
    const int n = P.n_ops, T = blockDim.x, tid = threadIdx.x;
    const int32_t per = (n + T - 1) / T;
    const int32_t kb = min(n, tid * per), ke = min(n, kb + per);
    // the thread's ops and their counts, each set of loads in one round
    int4 oi[kW];
    int32_t ck[kW];
#pragma unroll
    for (int j = 0; j < kW; ++j) oi[j] = kb + j < ke ? P.ord_info[kb + j] : make_int4(0, 0, 0, 0);
#pragma unroll
    for (int j = 0; j < kW; ++j) ck[j] = kb + j < ke ? __ldcg(&S.cnt[(int64_t)oi[j].x * kCntStride]) : 0;
    int32_t loc[3] = {0, 0, 0};
#pragma unroll
    for (int j = 0; j < kW; ++j) {
        if (kb + j >= ke) continue;
        int32_t f, t;
        op_tiles(ck[j], oi[j].y, min_vpl, ipt, kb + j >= P.n_cta_ops, f, t);
        loc[0] += ck[j];
        loc[1] += f;
        loc[2] += t;
    }
    int32_t excl[3], tot[3];
    block_scan3(loc, excl, tot, warp_sum);
    const int32_t tper = (n + nc - 1) / nc;
    const int32_t t0 = cb * tper, t1 = min(n, t0 + tper);
    int32_t pos = excl[0], tf = excl[1], tt = tot[1] + excl[2];
#pragma unroll
    for (int j = 0; j < kW; ++j) {
        const int k = kb + j;
        if (k >= ke) continue;
        const int32_t v = oi[j].x, nvec = oi[j].y, c = ck[j];
        op_start_s[v] = pos;
        if (k >= P.n_cta_ops) {
            if (k >= t0 && k < t1) {
                S.op_start[v] = pos;
                if (k == P.n_cta_ops) S.ctrl[kCtrlCtaTiles] = (unsigned long long)tt;
                write_warp_tiles(S, v, pos, c, ipt, make_int4(nvec * kVec, oi[j].w, oi[j].z, __ldg(P.ord_cbase + k)),
                                 tt);
            }
            tt += (c + 32 * ipt - 1) / (32 * ipt);
            pos += c;
            continue;
        }
        const int lg = lanes_log2_for(nvec, min_vpl);
        const int32_t per_tile = (kScoreThreads >> lg) * ipt;
        const int32_t full = full_tiles(c, lg, ipt), rest = c - full * per_tile;
        if (k >= t0 && k < t1) {
            S.op_start[v] = pos;  // for the count pass
            // {padded entries, distinct latencies, padded offset, first configuration}
            const int4 tx = make_int4(nvec * kVec, oi[j].w, oi[j].z, __ldg(P.ord_cbase + k));
            for (int32_t j = 0; j < full; ++j) {
                S.tiles[2 * (tf + j)] = make_int4(v, pos + j * per_tile, per_tile, lg);
                S.tiles[2 * (tf + j) + 1] = tx;
            }
            if (rest > 0) {
                S.tiles[2 * tt] = make_int4(v, pos + full * per_tile, rest, tail_lanes_log2(rest, lg, ipt, nvec));
                S.tiles[2 * tt + 1] = tx;
            }
        }
        tf += full;
        tt += rest > 0 ? 1 : 0;
        pos += c;
    }
    if (cb == 0 && tid == 0) {
        S.ctrl[kCtrlPositions] = (unsigned long long)tot[0];
        S.ctrl[kCtrlTiles] = (unsigned long long)(tot[1] + tot[2]);
    }
    __syncthreads();  // op_start_s complete
}

// All blocks of a cooperative launch reach this point before any continues.
// Bounded: after `tries` polls the block records a timeout and the barrier
// returns false in every thread of the block; the block must then stop (it
// does not arrive at later barriers, so every other block gives up at its next
// one).  The call's later kernels see the flag and decode nothing.
__device__ __forceinline__ bool grid_barrier(unsigned long long *count, unsigned long long target,
                                             unsigned long long *timeout, int32_t tries) {
    __syncthreads();
    int gave_up = 0;
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(count, 1ull);
        unsigned long long seen = 0;
        for (int it = 0; it < tries; ++it) {
            asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(seen) : "l"(count) : "memory");
            if (seen >= target) break;
        }
        if (seen < target) {
            atomicOr(timeout, 1ull);
            gave_up = 1;
        }
    }
    return !__syncthreads_or(gave_up);
}

// Nonzero once a bounded wait of the call gave up.  Read by the kernels that
// follow k_bucket after griddepcontrol.wait (k_bucket has completed and its
// writes are visible): they then read no bucket entry and no tile.
__device__ __forceinline__ bool call_timed_out(const BucketScratch &S) {
    return *reinterpret_cast<volatile unsigned long long *>(&S.ctrl[kCtrlTimeout]) != 0ull;
}

// Place invocation i in its op's bucket (op_start: first bucket position of
// every op) with its remaining time before queueing, max(0, SLO - elapsed)
// <= SLO < 2^31.  The scoring kernel turns it into the slack per backend
// (Algorithm 1 through the critical path); a non-positive remaining time gives
// slack 0 for every backend, since queueing times are >= 0.
__device__ __forceinline__ void scatter_invocation(const DevProblem &P, const BucketScratch &S,
                                                   const int32_t *op_start, int64_t i, int32_t g, int32_t slot,
                                                   int64_t rbase) {
    const int64_t pos = (int64_t)op_start[g] + slot;
    if (!LLAMA_IN_BOUNDS(P, pos >= 0 && pos < S.n_inv, LLAMA_CHECK_SCATTER)) return;
    S.b_ent[pos] = make_int2((int32_t)i, (int32_t)max(rbase, (int64_t)0));
}

// Validate and count a round of B invocations, i = i0 + j * stride for j < B
// (every load of the round is issued before any of its results is used, so a
// thread has B dependent chains in flight): g[j] = the global op (-1 if invalid,
// then its decision is written here, or if i >= n_inv), slot[j] = its rank in
// the op's bucket (one counter per 128-byte line, so concurrent atomics on
// different ops never share a line), rb[j] = target - elapsed time (Algorithm 1
// before the queueing time).  S.gop[i] is written for every invocation of the
// call; slot and rb also go to S.slot and S.rbase when store_rest (the caller
// does not keep them in registers).
template <int B>
__device__ __forceinline__ void count_round(const DevProblem &P, int64_t i0, int64_t stride, int64_t n_inv,
                                            const int32_t *dag, const int32_t *op_local, const int64_t *start,
                                            int64_t now, const BucketScratch &S, llama_decision *out,
                                            bool store_rest, int32_t (&g)[B], int32_t (&slot)[B],
                                            int64_t (&rb)[B]) {
    int32_t d[B], o[B];
    int64_t st[B];
#pragma unroll
    for (int j = 0; j < B; ++j) {
        const int64_t i = i0 + j * stride;
        const bool in = i < n_inv;
        d[j] = in ? dag[i] : -1;
        o[j] = in ? op_local[i] : 0;
        st[j] = in ? start[i] : 0;
    }
    // the checks of invocation_op, on each invocation's DAG record
    int4 di[B];
#pragma unroll
    for (int j = 0; j < B; ++j)
        di[j] = (d[j] >= 0 && d[j] < P.n_dags) ? __ldg(P.dag_info + d[j]) : make_int4(0, 0, 0, 0);
#pragma unroll
    for (int j = 0; j < B; ++j) {
        const bool ok = d[j] >= 0 && d[j] < P.n_dags && o[j] >= 0 && o[j] < di[j].y - di[j].x && st[j] >= 0 &&
                        st[j] <= now;
        g[j] = ok ? di[j].x + o[j] : -1;
        rb[j] = (int64_t)(((uint64_t)(uint32_t)di[j].w << 32) | (uint32_t)di[j].z) - (now - st[j]);
        slot[j] = ok ? atomicAdd(&S.cnt[(int64_t)g[j] * kCntStride], 1) : 0;
    }
#pragma unroll
    for (int j = 0; j < B; ++j) {
        const int64_t i = i0 + j * stride;
        if (i >= n_inv) continue;
        S.gop[i] = g[j];
        if (g[j] < 0) {
            llama_decision bad;
            bad.cfg = -1;
            bad.lat = 0;
            bad.cost = 0;
            bad.slack = 0;
            bad.flags = LLAMA_FLAG_INVALID;
            out[i] = bad;
            atomicAdd(&S.ctrl[kCtrlInvalid], 1ull);
        } else if (store_rest) {
            S.slot[i] = slot[j];
            S.rbase[i] = rb[j];
        }
    }
}

// Place a round of B invocations counted by count_round with store_rest (not
// kept in registers): their ops, slots and times loaded first, then the
// bucket starts, then the stores.
template <int B>
__device__ __forceinline__ void scatter_round(const DevProblem &P, const BucketScratch &S, const int32_t *op_start,
                                              int64_t i0, int64_t stride, int64_t n_inv) {
    int32_t g[B], sl[B];
    int64_t rb[B];
#pragma unroll
    for (int j = 0; j < B; ++j) {
        const int64_t i = i0 + j * stride;
        g[j] = i < n_inv ? S.gop[i] : -1;
    }
#pragma unroll
    for (int j = 0; j < B; ++j) {
        const int64_t i = i0 + j * stride;
        sl[j] = g[j] >= 0 ? S.slot[i] : 0;
        rb[j] = g[j] >= 0 ? S.rbase[i] : 0;
    }
    int32_t os[B];
#pragma unroll
    for (int j = 0; j < B; ++j) os[j] = g[j] >= 0 ? op_start[g[j]] : 0;
#pragma unroll
    for (int j = 0; j < B; ++j) {
        if (g[j] < 0) continue;
        const int64_t pos = (int64_t)os[j] + sl[j];
        if (!LLAMA_IN_BOUNDS(P, pos >= 0 && pos < S.n_inv, LLAMA_CHECK_SCATTER)) continue;
        S.b_ent[pos] = make_int2((int32_t)(i0 + j * stride), (int32_t)max(rb[j], (int64_t)0));
    }
}

// The bucketing step of a call, one cooperative launch (all blocks resident,
// four per SM at 64 registers):
//  1. blocks [0, n_cp) compute the critical paths (a warp per small DAG); the
//     other blocks validate invocations, count them per op (one counter per
//     128-byte line, so concurrent atomics on different ops never share a
//     line), in rounds of kRound per thread after the first kKeep, and
//     prefetch the encoded tables into L2;
//  2. the counting blocks lay out the buckets and the scoring tiles, ops in
//     the order P.op_order (largest tables first), every op's full tiles
//     first, then the tails: per-block sums, a barrier of the counting
//     blocks, prefixes over the blocks and the writes;
//  3. grid barrier;
//  4. the counting blocks place their invocations in their buckets, each with
//     its remaining time (the scoring kernel turns it into the slack per
//     backend, Algorithm 1 through the critical path).
__global__ void __launch_bounds__(256, 4) k_bucket(DevProblem P, int64_t n_inv, const int32_t *dag,
                                                const int32_t *op_local, const int64_t *start,
                                                int64_t now, BucketScratch S, llama_decision *out,
                                                const int32_t *topo, const int32_t *lvl_off,
                                                const int32_t *dag_lvl, int32_t min_vpl, int32_t ipt,
                                                int32_t n_cp) {
    __shared__ int32_t warp_sum[3][32];
    __shared__ CpSmem sm;
    {
        // one parallel round of L2 prefetches of every small array the dependent
        // load chains below will touch (each line starts inside its array)
        int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        const int64_t step = (int64_t)gridDim.x * blockDim.x;
#pragma unroll 1
        for (int a = 0; a < kPfArrays; ++a) {
            for (; l < P.pf_lines[a]; l += step)
                asm volatile("prefetch.global.L2::evict_last [%0];" ::"l"(P.pf_ptr[a] + 128 * l));
            l -= P.pf_lines[a];
        }
    }
    if ((int)blockIdx.x < n_cp) {
        // nothing in this kernel waits for the critical paths: the scoring
        // kernel reads them after griddepcontrol.wait
        critical_paths_of_block(P, blockIdx.x, n_cp, topo, lvl_off, dag_lvl, sm);
        return;
    }
    // counting blocks: each thread takes invocations base, base + stride, ...;
    // the first kKeep of them stay in registers (op, slot in the bucket,
    // remaining time before queueing) across the grid barrier
    const int64_t nb = gridDim.x - n_cp;
    const int64_t stride = nb * blockDim.x;
    const int64_t base = (blockIdx.x - n_cp) * (int64_t)blockDim.x + threadIdx.x;
    int32_t kg[kKeep], ks[kKeep];
    int64_t kr[kKeep];
    count_round<kKeep>(P, base, stride, n_inv, dag, op_local, start, now, S, out, false, kg, ks, kr);
    for (int64_t i0 = base + kKeep * stride; i0 < n_inv; i0 += kRound * stride) {
        int32_t g[kRound], sl[kRound];
        int64_t rb[kRound];
        count_round<kRound>(P, i0, stride, n_inv, dag, op_local, start, now, S, out, true, g, sl, rb);
    }
    // Pull the encoded tables into L2 while the buckets are laid out, so the
    // scoring kernel's staging does not wait on DRAM.
    if (P.prefetch_rank_lines > 0) {
        // lrb, rf (, df): 2*n_pad bytes each; dlat: 4*n_pad bytes; every
        // prefetched line starts inside its array
        const char *arr[3] = {reinterpret_cast<const char *>(P.lrb), reinterpret_cast<const char *>(P.rf),
                              reinterpret_cast<const char *>(P.df)};
        const int n_arr = P.df ? 3 : 2;
        const int64_t n_rank = P.prefetch_rank_lines * n_arr;
        for (int64_t l = base; l < n_rank + P.prefetch_dlat_lines; l += stride) {
            const char *a = l < n_rank ? arr[l % n_arr] + 128 * (l / n_arr)
                                       : reinterpret_cast<const char *>(P.dlat) + 128 * (l - n_rank);
            asm volatile("prefetch.global.L2::evict_last [%0];" ::"l"(a));
        }
    }
    // the counting blocks lay out the buckets and tiles (the critical-path
    // blocks do not take part): once the counts are final, either every block
    // computes the whole layout itself (bucket starts in shared memory, in the
    // critical-path staging area these blocks do not use), or, for more ops,
    // per-block sums, prefixes over the blocks and the writes between two more
    // barriers of the counting blocks
    // A barrier that gives up ends the block: counts that are not final give
    // no layout, and a layout that is not complete no scatter.
    const int32_t cb = (int32_t)(blockIdx.x - n_cp);
    unsigned long long *const bar = &S.ctrl[kCtrlCountBarrier], *const tmo = &S.ctrl[kCtrlTimeout];
    if (!grid_barrier(bar, (unsigned long long)nb, tmo, P.wait_tries)) return;
    const int32_t *op_start;
    if (P.n_ops <= kLayoutWholeOps) {
        int32_t *op_start_s = reinterpret_cast<int32_t *>(&sm);
        layout_whole(P, S, cb, (int32_t)nb, min_vpl, ipt, op_start_s, warp_sum);
        op_start = op_start_s;
    } else {
        LayoutRun R;
        layout_sums(P, S, cb, (int32_t)nb, min_vpl, ipt, R, warp_sum);
        if (!grid_barrier(bar, 2ull * (unsigned long long)nb, tmo, P.wait_tries)) return;
        layout_write(P, S, cb, (int32_t)nb, min_vpl, ipt, R, warp_sum);
        if (!grid_barrier(bar, 3ull * (unsigned long long)nb, tmo, P.wait_tries)) return;
        op_start = S.op_start;
    }

    // let the scoring kernel start staging its tables while the scatter runs
    asm volatile("griddepcontrol.launch_dependents;");
#pragma unroll
    for (int j = 0; j < kKeep; ++j)
        if (kg[j] >= 0) scatter_invocation(P, S, op_start, base + j * stride, kg[j], ks[j], kr[j]);
    for (int64_t i0 = base + kKeep * stride; i0 < n_inv; i0 += kRound * stride)
        scatter_round<kRound>(P, S, op_start, i0, stride, n_inv);
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
        for (int h = 0; h < H; ++h)
            slack_out[i * H + h] = slack_of(P.ref[g], P.cp[g], P.cp_magic[g], r_base - P.q[h]);
    }
}

// ---------------------------------------------------------------------------
// a4: scoring
// ---------------------------------------------------------------------------

// Eight configurations of one segment, for an invocation whose slack has c
// distinct latencies of the op below it (c2 = c in both halves).  lk holds
// 0x8000 + latency rank of each config: lk - c2 subtracts per 16-bit half
// without borrow (ranks and c are below 8192), and bit 15 of a half is set
// exactly when rank >= c, i.e. L >= slack (infeasible).  Cost-first: those
// bits are OR-ed onto the feasible-branch ranks (an infeasible key is >=
// 0x8000, above every feasible one); alpha: they are replicated into a 0xFFFF
// mask that selects the infeasible-branch rank rf ^ df.  Then a per-half
// unsigned 16-bit running minimum.
__device__ __forceinline__ uint32_t scan8_cost_first(uint32_t best, uint32_t c2, uint4 lk, uint4 rk) {
    best = vmin_u16x2(best, rk.x | ((lk.x - c2) & 0x80008000u));
    best = vmin_u16x2(best, rk.y | ((lk.y - c2) & 0x80008000u));
    best = vmin_u16x2(best, rk.z | ((lk.z - c2) & 0x80008000u));
    best = vmin_u16x2(best, rk.w | ((lk.w - c2) & 0x80008000u));
    return best;
}

__device__ __forceinline__ uint32_t scan8_alpha(uint32_t best, uint32_t c2, uint4 lk, uint4 rk, uint4 dk) {
    best = vmin_u16x2(best, rk.x ^ (dk.x & prmt(lk.x - c2, 0, 0xBB99u)));
    best = vmin_u16x2(best, rk.y ^ (dk.y & prmt(lk.y - c2, 0, 0xBB99u)));
    best = vmin_u16x2(best, rk.z ^ (dk.z & prmt(lk.z - c2, 0, 0xBB99u)));
    best = vmin_u16x2(best, rk.w ^ (dk.w & prmt(lk.w - c2, 0, 0xBB99u)));
    return best;
}

// Number of values below s in the ascending array d[0..m); d may point to
// shared or global memory (generic loads).
__device__ __forceinline__ int32_t count_below(const int32_t *d, int32_t m, int32_t s) {
    int32_t lo = 0, hi = m;
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (d[mid] < s) lo = mid + 1; else hi = mid;
    }
    return lo;
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

// A tile is (op, first bucket position, m invocations, 2^lg lanes per group).
// For a tile, the op's encoded table is staged into shared memory by TMA bulk
// copies, in chunks of at most `chunk` entries (a multiple of 8); the lanes
// count, for each invocation and segment, the op's distinct latencies below
// the slack.  A group of 2^lg lanes scores IPT consecutive invocations: lane s
// takes the vectors q = s mod 2^lg of every backend segment, loads each vector
// once from shared memory and applies it to all IPT invocations, each against
// its own count for that segment.  Groups reduce with shuffles (and through
// shared memory when a group spans several warps); lane u mod 2^lg of a group
// decodes the group's invocation u.

// Start of a scoring kernel, once the bucketing kernel's results are visible:
// its per-op counters are no longer read, so they are cleared for the next call.
__device__ __forceinline__ void clear_counters(const DevProblem &P, const BucketScratch &S) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P.n_ops;
         k += (int64_t)gridDim.x * blockDim.x)
        S.cnt[k * kCntStride] = 0;
}

// End of a scoring kernel: the last CTA to finish publishes the call's status
// and clears the control words, so the next call needs no memset.  If a
// bounded wait of the call gave up (bucketing barrier or table staging), that
// CTA first marks every valid invocation not decided (cfg = -1,
// LLAMA_FLAG_TIMEOUT): every other CTA has finished, so nothing overwrites
// them, and decisions of tiles scored before the wait gave up are dropped too.
// Invalid invocations keep what k_bucket wrote.  S.gop was written for every
// invocation of the call before k_bucket's first barrier; k_stair (mark =
// false) writes no S.gop and has no bounded wait.
__device__ __forceinline__ void finish_call(const BucketScratch &S, llama_decision *out, bool mark) {
    __shared__ int role;  // 0: not the last CTA; 1: the last; 2: the last, and the call timed out
    __syncthreads();
    if (threadIdx.x == 0) {
        role = 0;
        __threadfence();
        if (atomicAdd(&S.ctrl[kCtrlDone], 1ull) == (unsigned long long)gridDim.x - 1) {
            __threadfence();
            const unsigned long long tmo = atomicAdd(&S.ctrl[kCtrlTimeout], 0ull);
            S.status[0] = atomicAdd(&S.ctrl[kCtrlInvalid], 0ull);
            S.status[1] = tmo;
            role = tmo && mark ? 2 : 1;
        }
    }
    __syncthreads();
    if (role == 2) {  // block-uniform
        llama_decision nd;
        nd.cfg = -1;
        nd.lat = 0;
        nd.cost = 0;
        nd.slack = 0;
        nd.flags = LLAMA_FLAG_TIMEOUT;
        for (int64_t i = threadIdx.x; i < S.n_inv; i += blockDim.x)
            if (__ldcg(&S.gop[i]) >= 0) out[i] = nd;
        __syncthreads();
    }
    if (role != 0 && threadIdx.x == 0)
        for (int k = 0; k < kCtrlWords; ++k) atomicExch(&S.ctrl[k], 0ull);
}

// Per-thread view of the current tile.
template <int IPT>
struct TileState {
    int32_t v, m, lg, L, g, s, npad, dn;
    int32_t pos0;  // bucket position of the group's first invocation
    int32_t cbase;  // cfg_off of the op
    int64_t p0;
    int32_t inv[IPT];
    uint32_t best[IPT];
    bool any;
    // the op's reference latency, critical path and floor((2^64-1) / critical
    // path), loaded by every thread as the tile starts (one request per warp;
    // nothing waits for them before the table copy is issued)
    int64_t ref, cp;
    uint64_t mg;
};

// The queueing time per backend, copied into shared memory once per call.
struct TileConst {
    int64_t q[LLAMA_MAX_HW];
};

template <int IPT>
__device__ __forceinline__ void tile_begin(const DevProblem &P, const BucketScratch &S, long long ti,
                                           TileConst &tc, TileState<IPT> &T) {
    const int4 tile = S.tiles[2 * ti], tx = S.tiles[2 * ti + 1];
    T.v = tile.x;
    T.m = tile.z;
    T.lg = tile.w;
    T.L = 1 << T.lg;
    T.g = threadIdx.x >> T.lg;
    T.s = threadIdx.x & (T.L - 1);
    T.npad = tx.x;
    T.dn = tx.y;
    T.p0 = tx.z;
    T.cbase = tx.w;
    T.any = false;
    T.pos0 = tile.y + T.g * IPT;
#pragma unroll
    for (int u = 0; u < IPT; ++u) {
        const int32_t j = T.g * IPT + u;
        const bool in = j < T.m && LLAMA_IN_BOUNDS(P, tile.y + j >= 0 && tile.y + j < S.n_inv, LLAMA_CHECK_TILE);
        T.inv[u] = in ? S.b_ent[tile.y + j].x : -1;
        if (!LLAMA_IN_BOUNDS(P, T.inv[u] < S.n_inv, LLAMA_CHECK_TILE)) T.inv[u] = -1;
        T.any |= T.inv[u] >= 0;
        T.best[u] = 0xFFFFFFFFu;
    }
    T.ref = P.ref[T.v];
    T.cp = P.cp[T.v];
    T.mg = P.cp_magic[T.v];
}

// inv[u] for a runtime u, without a runtime index into registers.
template <int IPT>
__device__ __forceinline__ int32_t inv_at(const TileState<IPT> &T, int u) {
    int32_t iu = T.inv[0];
#pragma unroll
    for (int w = 1; w < IPT; ++w) iu = u == w ? T.inv[w] : iu;
    return iu;
}

// Slack of the tile's invocation u for backend h: Algorithm 1 through the
// critical path, floor(ref * (rem - Q[h]) / cp), 0 once the target has passed,
// rem being the invocation's remaining time stored beside its bucket entry.
template <int IPT>
__device__ __forceinline__ int32_t slack_at(const BucketScratch &S, const TileState<IPT> &T, const TileConst &tc,
                                            int u, int h) {
    return slack_of(T.ref, T.cp, T.mg, (int64_t)S.b_ent[T.pos0 + u].y - tc.q[h]);
}

// Counts c(u, h) of distinct latencies below the slack of invocation u for
// backend h, into cg[u * H + h], from the sorted list dl (shared memory: the
// lanes of a group share the bisections).
template <int IPT>
__device__ __forceinline__ void counts_from_shared(const BucketScratch &S, const TileState<IPT> &T,
                                                   const TileConst &tc, int H, const int32_t *dl, uint16_t *cg) {
    if (!T.any) return;
    for (int t = T.s; t < IPT * H; t += T.L) {
        const int u = t / H, h = t - u * H;
        const int32_t iu = inv_at(T, u);
        cg[t] = iu >= 0 ? (uint16_t)count_below(dl, T.dn, slack_at(S, T, tc, u, h)) : 0;
    }
}

// The same counts from the list in global memory: each search is shared by
// G <= 32 lanes, a G-ary search (a few dependent rounds instead of log2 dn).
// A round over n > G candidates [lo, lo + n) probes lo + (l+1)n/G - 1 for
// l < G (strictly increasing, the last one at lo + n - 1); over n <= G
// candidates it probes each one.  Only shifts: G is a power of two and
// (l+1)n < 2^19.  Every thread of the CTA must call this (warp votes).
template <int IPT>
__device__ __forceinline__ void counts_from_global(const DevProblem &P, const BucketScratch &S,
                                                   const TileState<IPT> &T, const TileConst &tc, int H,
                                                   const int32_t *dl, uint16_t *cg) {
    const int nc = IPT * H;
    const int G = T.L < 32 ? T.L : 32, lgG = T.lg < 5 ? T.lg : 5;
    const int W = T.L > 32 ? (T.L >> 5) : 1, sw = T.s >> 5, gl = T.s & (G - 1);
    const int gbase = (threadIdx.x & 31) & ~(G - 1);
    const uint32_t gmask = G == 32 ? 0xFFFFFFFFu : ((1u << G) - 1u);
    for (int t0 = 0; t0 < nc; t0 += W) {
        const int t = t0 + sw, u = t / H, h = t - u * H;
        const int32_t iu = inv_at(T, u);
        const bool act = t < nc && iu >= 0;
        const int32_t sl = act ? slack_at(S, T, tc, u, h) : 0;
        int32_t lo = 0, hi = act ? T.dn : 0;  // lo <= count <= hi
        if (G == 1) {  // one lane per invocation (tile-uniform): bisection
            lo = hi = act ? count_below(dl, T.dn, sl) : 0;
        }
        while (__any_sync(0xFFFFFFFFu, hi > lo)) {
            const int32_t n = hi - lo;
            const bool exact = n <= G;
            const int32_t pos = exact ? lo + gl : lo + (((gl + 1) * n) >> lgG) - 1;
            bool pred = false;
            if (n > 0 && (!exact || gl < n)) {
                // a 32-lane first round reads the op's probe values from one line
                const bool first = G == 32 && !exact && n == T.dn;
                pred = (first ? __ldg(P.dpiv + 32 * (int64_t)T.v + gl) : __ldg(dl + pos)) < sl;
            }
            const int32_t c = __popc((__ballot_sync(0xFFFFFFFFu, pred) >> gbase) & gmask);
            if (n > 0) {
                if (exact) {
                    lo += c;
                    hi = lo;
                } else {
                    // the answer lies after the last probe below sl and at or
                    // before the first one that is not
                    const int32_t nhi = c < G ? lo + (((c + 1) * n) >> lgG) - 1 : hi;
                    lo = c > 0 ? lo + ((c * n) >> lgG) : lo;
                    hi = nhi;
                }
            }
        }
        if (act && gl == 0) cg[t] = (uint16_t)lo;
    }
}

// The counts of the tile's invocations computed by the count pass (k_counts):
// c_s[j * H + h] = b_cnt[(b0 + j) * H + h] for the tile's j-th invocation,
// which is cg[u * H + h] of the group holding j = g * IPT + u.  Every thread of
// the CTA must call this; a block barrier must separate it from the reads.
template <int IPT>
__device__ __forceinline__ void counts_from_pass(const BucketScratch &S, const TileState<IPT> &T, int H,
                                                 uint16_t *c_s) {
    const int nc = T.m * H;
    const uint16_t *src = S.b_cnt + (int64_t)(T.pos0 - T.g * IPT) * H;
    for (int t = threadIdx.x; t < nc; t += kScoreThreads) c_s[t] = src[t];
}

// Score the staged chunk [c0, c0 + cn) of the tile's op.
template <int MODE, int IPT>
__device__ __forceinline__ void scan_chunk(const DevProblem &P, TileState<IPT> &T, int32_t c0, int32_t cn,
                                           const uint16_t *lr_s, const uint16_t *rf_s, const uint16_t *df_s,
                                           const uint16_t *cg) {
    if (!T.any) return;
    const int H = P.n_hw;
    const int32_t *sp = P.seg_pad + (int64_t)T.v * (H + 1);
    const int qc0 = c0 / kVec, qc1 = (c0 + cn) / kVec;
    const uint4 *lr4 = reinterpret_cast<const uint4 *>(lr_s);
    const uint4 *rf4 = reinterpret_cast<const uint4 *>(rf_s);
    const uint4 *df4 = reinterpret_cast<const uint4 *>(df_s);
    for (int h = 0; h < H; ++h) {
        const int a = max(__ldg(sp + h) / kVec, qc0), b = min(__ldg(sp + h + 1) / kVec, qc1);
        if (a >= b) continue;
        uint32_t c2[IPT];
#pragma unroll
        for (int u = 0; u < IPT; ++u) c2[u] = (uint32_t)cg[u * H + h] * 0x00010001u;
        for (int q = a + ((T.s - a) & (T.L - 1)); q < b; q += T.L) {
            const int r = q - qc0;
            const uint4 lk = lr4[r], rk = rf4[r];
            if (MODE == LLAMA_MODE_ALPHA) {
                const uint4 dk = df4[r];
#pragma unroll
                for (int u = 0; u < IPT; ++u) T.best[u] = scan8_alpha(T.best[u], c2[u], lk, rk, dk);
            } else {
#pragma unroll
                for (int u = 0; u < IPT; ++u) T.best[u] = scan8_cost_first(T.best[u], c2[u], lk, rk);
            }
        }
    }
}

// The decision of one invocation of op v (first configuration cbase) from its
// least key, and its slack on the chosen backend (Algorithm 1 from the
// remaining time rem), into *dst.
template <int MODE>
__device__ __forceinline__ void decode_into(const DevProblem &P, int32_t v, int32_t cbase, uint32_t key,
                                            int64_t ref, int64_t cp, uint64_t mg, int64_t rem,
                                            const TileConst &tc, llama_decision *dst) {
    if (!LLAMA_IN_BOUNDS(P, decode_key_ok(P, v, key, MODE), LLAMA_CHECK_DECODE)) return;
    int4 d;
    if (MODE == LLAMA_MODE_ALPHA) d = P.dec[2 * (int64_t)cbase + key];
    else d = key < 0x8000u ? P.dec[(int64_t)cbase + key] : P.dfast[v];
    const int32_t sl = slack_of(ref, cp, mg, rem - tc.q[d.x >> 16]);
    llama_decision dsn;
    dsn.cfg = d.x & 0xFFFF;
    dsn.lat = d.y;
    dsn.cost = (int64_t)(((uint64_t)(uint32_t)d.w << 32) | (uint32_t)d.z);
    dsn.slack = sl;
    dsn.flags = d.y < sl ? LLAMA_FLAG_FEASIBLE : 0;
    *dst = dsn;
}

// Reduce each group's keys and decode them into decisions.  Every thread of
// the CTA must call this (a block barrier when groups span several warps).
template <int MODE, int IPT>
__device__ __forceinline__ void finish_tile(const DevProblem &P, const BucketScratch &S, llama_decision *out,
                                            const TileState<IPT> &T, const TileConst &tc,
                                            uint32_t (*red)[kScoreThreads / 32]) {
    const int tid = threadIdx.x;
    uint32_t key[IPT];
    const int wl = T.L < 32 ? T.L : 32;
#pragma unroll
    for (int u = 0; u < IPT; ++u) {
        key[u] = T.inv[u] >= 0 ? min(T.best[u] & 0xFFFFu, T.best[u] >> 16) : 0xFFFFu;
        for (int o = 1; o < wl; o <<= 1) key[u] = min(key[u], __shfl_xor_sync(0xffffffffu, key[u], o));
    }
    if (T.L > 32) {
        // a group spans L/32 warps: combine the warps' minima in shared memory
        if ((tid & 31) == 0)
            for (int u = 0; u < IPT; ++u) red[u][tid >> 5] = key[u];
        __syncthreads();
        if (T.s < IPT)  // the decoding lanes (L > 32 > IPT here)
            for (int u = 0; u < IPT; ++u)
                for (int w = 1; w < (T.L >> 5); ++w) key[u] = min(key[u], red[u][(tid >> 5) + w]);
    }
    // lane u mod 2^lg of the group decodes invocation u (every lane holds every key)
#pragma unroll
    for (int u = 0; u < IPT; ++u) {
        if (T.s != (u & (T.L - 1)) || T.inv[u] < 0) continue;
        decode_into<MODE>(P, T.v, T.cbase, key[u], T.ref, T.cp, T.mg, (int64_t)S.b_ent[T.pos0 + u].y, tc,
                          out + T.inv[u]);
    }
}

// Queue the bulk copies of chunk [c0, c0 + cn) of the table at padded offset
// p0 (and, with the first chunk, the op's dn distinct latencies when they are
// staged) on mbarrier bar.  One thread.
template <int MODE>
__device__ __forceinline__ void stage_chunk(const DevProblem &P, int64_t p0, int32_t c0, int32_t cn,
                                            bool with_dlat, int32_t dn, uint16_t *lr_s, uint16_t *rf_s,
                                            uint16_t *df_s, int32_t *dl_s, uint32_t bar) {
    // the generic-proxy reads of this buffer are complete (a block barrier came
    // before); order them before the async-proxy writes that follow
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    // whole 16-byte words of the distinct latencies: dlat has npad >= dn entries here
    const uint32_t db = with_dlat ? (uint32_t)((dn + 3) / 4) * 16u : 0u;
    // checked build: a range outside the padded tables is not copied (the
    // mbarrier still completes, with no bytes expected)
    if (!LLAMA_IN_BOUNDS(P, p0 >= 0 && c0 >= 0 && p0 + c0 + cn <= P.n_pad && p0 + (int64_t)db / 4 <= P.n_pad,
                         LLAMA_CHECK_STAGE)) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(0u) : "memory");
        return;
    }
    const uint32_t bytes = (uint32_t)cn * (MODE == LLAMA_MODE_ALPHA ? 6u : 4u) + db;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    if (with_dlat) bulk_g2s(dl_s, P.dlat + p0, db, bar);
    bulk_g2s(lr_s, P.lrb + p0 + c0, 2u * cn, bar);
    bulk_g2s(rf_s, P.rf + p0 + c0, 2u * cn, bar);
    if (MODE == LLAMA_MODE_ALPHA) bulk_g2s(df_s, P.df + p0 + c0, 2u * cn, bar);
}

__device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Bring [src, src + bytes) into L2 (16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void prefetch_l2(const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<uint64_t>(src)), "r"(bytes)
                 : "memory");
}

// The warp tiles [n_cta, n_tiles), after the CTA's last whole-CTA tile: each
// warp takes them one at a time from a counter (the next claim in flight
// while a tile is scored), with no block barrier, so up to kScoreWarps tiles
// per CTA progress independently.  A warp copies the op's rank vectors and
// distinct latencies into its own kWarpSlice bytes of shared memory with
// 16-byte loads; lane l takes the tile's invocations l * IPT + u (u < IPT,
// below m).  Per backend segment, each lane counts the distinct latencies
// below each of its slacks (a bisection of the staged list), then every lane
// scans the same vectors of the segment (broadcast reads), as scan_chunk does
// with one lane per group; each lane then decodes its invocations.  Every
// thread of the CTA calls this after a block barrier (the whole-CTA staging
// buffers are free: no copy in flight).
template <int MODE, int IPT>
__device__ __forceinline__ void warp_tiles(const DevProblem &P, const BucketScratch &S, llama_decision *out,
                                           unsigned char *smem_raw, long long n_cta, long long n_tiles,
                                           const TileConst &tc) {
    constexpr int kTb = MODE == LLAMA_MODE_ALPHA ? 6 : 4;  // staged bytes per table entry
    const int H = P.n_hw, lane = threadIdx.x & 31;
    unsigned char *slice = smem_raw + (size_t)(threadIdx.x >> 5) * kWarpSlice;
    unsigned long long claim = 0;
    if (lane == 0) claim = atomicAdd(&S.ctrl[kCtrlNextWarpTile], 1ull);
    long long wt = n_cta + (long long)__shfl_sync(0xffffffffu, claim, 0);
    while (wt < n_tiles) {
        if (lane == 0) claim = atomicAdd(&S.ctrl[kCtrlNextWarpTile], 1ull);  // the tile after this one
        const int4 tile = S.tiles[2 * wt], tx = S.tiles[2 * wt + 1];
        const int32_t v = tile.x, m = tile.z, npad = tx.x, dn = tx.y, cbase = tx.w;
        const int64_t p0 = tx.z;
        // tables at padded offsets (multiples of 8 entries: 16-byte aligned);
        // the distinct latencies after the table (npad * kTb is a multiple of 16)
        const bool fits = LLAMA_IN_BOUNDS(P, p0 >= 0 && p0 + npad <= P.n_pad && (size_t)npad * (kTb + 4) <= kWarpSlice &&
                                                 dn <= npad && tile.y >= 0 && tile.y + m <= S.n_inv,
                                          LLAMA_CHECK_TILE);
        uint4 *lr4 = reinterpret_cast<uint4 *>(slice);
        uint4 *rf4 = lr4 + npad / kVec;
        uint4 *df4 = rf4 + npad / kVec;
        int32_t *dl_s = reinterpret_cast<int32_t *>(slice + (size_t)npad * kTb);
        if (fits) {
            const uint4 *glr = reinterpret_cast<const uint4 *>(P.lrb + p0);
            const uint4 *grf = reinterpret_cast<const uint4 *>(P.rf + p0);
            const uint4 *gdf = reinterpret_cast<const uint4 *>(P.df + p0);
            for (int k = lane; k < npad / kVec; k += 32) {
                lr4[k] = __ldg(glr + k);
                rf4[k] = __ldg(grf + k);
                if (MODE == LLAMA_MODE_ALPHA) df4[k] = __ldg(gdf + k);
            }
            const int4 *gdl = reinterpret_cast<const int4 *>(P.dlat + p0);
            for (int k = lane; k < (dn + 3) / 4; k += 32) reinterpret_cast<int4 *>(dl_s)[k] = __ldg(gdl + k);
        }
        int32_t inv[IPT];
        int64_t rem[IPT];
        uint32_t best[IPT];
#pragma unroll
        for (int u = 0; u < IPT; ++u) {
            const int32_t j = lane * IPT + u;
            const bool in = fits && j < m;
            const int2 e = in ? S.b_ent[tile.y + j] : make_int2(-1, 0);
            inv[u] = e.x;
            if (!LLAMA_IN_BOUNDS(P, inv[u] < S.n_inv, LLAMA_CHECK_TILE)) inv[u] = -1;
            rem[u] = e.y;
            best[u] = 0xFFFFFFFFu;
        }
        const int64_t ref = P.ref[v], cp = P.cp[v];
        const uint64_t mg = P.cp_magic[v];
        const int32_t *sp = P.seg_pad + (int64_t)v * (H + 1);
        __syncwarp();
        for (int h = 0; fits && h < H; ++h) {
            const int a = __ldg(sp + h) / kVec, b = __ldg(sp + h + 1) / kVec;
            if (a >= b) continue;
            uint32_t c2[IPT];
#pragma unroll
            for (int u = 0; u < IPT; ++u)
                c2[u] = inv[u] >= 0 ? (uint32_t)count_below(dl_s, dn, slack_of(ref, cp, mg, rem[u] - tc.q[h])) *
                                          0x00010001u
                                    : 0u;
            for (int q = a; q < b; ++q) {
                const uint4 lk = lr4[q], rk = rf4[q];
                if (MODE == LLAMA_MODE_ALPHA) {
                    const uint4 dk = df4[q];
#pragma unroll
                    for (int u = 0; u < IPT; ++u) best[u] = scan8_alpha(best[u], c2[u], lk, rk, dk);
                } else {
#pragma unroll
                    for (int u = 0; u < IPT; ++u) best[u] = scan8_cost_first(best[u], c2[u], lk, rk);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < IPT; ++u)
            if (inv[u] >= 0)
                decode_into<MODE>(P, v, cbase, min(best[u] & 0xFFFFu, best[u] >> 16), ref, cp, mg, rem[u], tc,
                                  out + inv[u]);
        __syncwarp();  // every lane is done with the slice before the next tile is copied in
        wt = n_cta + (long long)__shfl_sync(0xffffffffu, claim, 0);
    }
}

// One staging buffer.  Persistent CTAs take tiles from the tile list: first
// tile blockIdx.x, the next ones from an atomic counter, so CTAs that finish
// early take more (the list is ordered longest first).  While the first chunk
// lands, the distinct latencies are searched.  The next tile is claimed as a
// tile starts and its descriptor read while the tile's copy lands, so its
// first chunk is copied as soon as the scan is done with the buffer, while
// this tile's decisions are decoded.
template <int MODE, int IPT, bool WARP>
__device__ __forceinline__ void score_body(const DevProblem &P, const BucketScratch &S,
                                           llama_decision *out, int32_t chunk, int32_t dl_cap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // chunk entries: latency ranks, feasible-branch ranks (, rank differences);
    // the op's distinct latencies; per group, the counts of each invocation
    uint16_t *lr_s = reinterpret_cast<uint16_t *>(smem_raw);
    uint16_t *rf_s = lr_s + chunk;
    uint16_t *df_s = rf_s + chunk;
    const size_t tbl = align16((size_t)chunk * (MODE == LLAMA_MODE_ALPHA ? 6 : 4));
    int32_t *dl_s = reinterpret_cast<int32_t *>(smem_raw + tbl);
    uint16_t *c_s = reinterpret_cast<uint16_t *>(smem_raw + tbl + 4 * (size_t)dl_cap);
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ uint32_t red[IPT][kScoreThreads / 32];
    __shared__ long long next_tile;
    __shared__ TileConst tc;
    const int tid = threadIdx.x, H = P.n_hw;
    const uint32_t bar = smem_addr(&mbar);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t phase = 0;
    bool ok = true;
    // everything k_bucket wrote (tile list, buckets, slack) is visible only after
    // griddepcontrol.wait; the mbarrier set-up above overlaps its tail
    asm volatile("griddepcontrol.wait;" ::: "memory");
    clear_counters(P, S);
    if (tid < H) tc.q[tid] = P.q[tid];
    // after a bucketing barrier gave up, no tile list or bucket entry is read
    const long long n_tiles = call_timed_out(S) ? 0 : (long long)S.ctrl[kCtrlTiles];
    // the whole-CTA tiles come first; the warp tiles after them (a kernel
    // without the warp phase scores any warp tile as a CTA tile of one lane
    // per invocation, with the same result)
    const long long n_cta =
        WARP && P.n_cta_ops < P.n_ops ? min((long long)S.ctrl[kCtrlCtaTiles], n_tiles) : n_tiles;
    long long ti = blockIdx.x;
    // the first chunk of a tile, from the tile's descriptor tx = {npad, dn, p0}
    // (every op has at least one configuration: npad > 0)
    const auto first_chunk = [&](const int4 &tx) {
        stage_chunk<MODE>(P, (int64_t)tx.z, 0, min(chunk, tx.x), tx.y <= dl_cap, tx.y, lr_s, rf_s, df_s, dl_s, bar);
    };
    if (ti < n_cta && tid == 0) first_chunk(S.tiles[2 * ti + 1]);
    bool pending = ti < n_cta;  // a copy into the buffer is in flight
    __syncthreads();
    TileState<IPT> T;
    while (ti < n_cta) {
        unsigned long long claim = 0;
        if (tid == 0) claim = atomicAdd(&S.ctrl[kCtrlNextTile], 1ull);  // the tile after this one
        tile_begin(P, S, ti, tc, T);
        const bool dl_staged = T.dn <= dl_cap;
        uint16_t *cg = c_s + T.g * IPT * H;
        int4 txn = make_int4(0, 0, 0, 0);
        for (int32_t c0 = 0; c0 < T.npad; c0 += chunk) {
            const int32_t cn = min(chunk, T.npad - c0);
            if (c0 > 0) {
                __syncthreads();  // every thread is done with the previous chunk
                if (tid == 0) stage_chunk<MODE>(P, T.p0, c0, cn, false, T.dn, lr_s, rf_s, df_s, dl_s, bar);
                pending = true;
            }
            if (c0 == 0 && !dl_staged) {
                if (S.b_cnt) counts_from_pass(S, T, H, c_s);
                else counts_from_global(P, S, T, tc, H, P.dlat + T.p0, cg);
            }
            // every thread must agree before any leaves the barrier sequence
            if (!__syncthreads_and(mbar_wait(bar, phase))) {
                ok = false;
                break;
            }
            phase ^= 1u;
            pending = false;
            if (c0 == 0) {
                if (tid == 0) {
                    const long long tn = (long long)(claim + gridDim.x);
                    next_tile = tn;
                    if (tn < n_cta) {
                        // the next tile's first chunk goes to L2 while this one is scored
                        txn = S.tiles[2 * tn + 1];
                        const uint32_t pb = 2u * (uint32_t)min(chunk, txn.x);
                        prefetch_l2(P.lrb + txn.z, pb);
                        prefetch_l2(P.rf + txn.z, pb);
                        if (MODE == LLAMA_MODE_ALPHA) prefetch_l2(P.df + txn.z, pb);
                    }
                }
                if (dl_staged) {
                    counts_from_shared(S, T, tc, H, dl_s, cg);
                    __syncthreads();
                }
            }
            scan_chunk<MODE, IPT>(P, T, c0, cn, lr_s, rf_s, df_s, cg);
        }
        if (!ok) break;
        __syncthreads();  // the scan is done with the buffer; next_tile is published
        const long long tn = next_tile;
        if (tn < n_cta) {
            if (tid == 0) first_chunk(txn);
            pending = true;
        }
        finish_tile<MODE, IPT>(P, S, out, T, tc, red);
        ti = tn;
    }
    if (!ok || pending) {
        // a staging copy never completed: report it, wait (bounded) for the copy
        // to land so no transfer targets this CTA's shared memory after exit
        if (!ok && tid == 0) atomicOr(&S.ctrl[kCtrlTimeout], 1ull);
        mbar_wait(bar, phase);
    }
    if (WARP && ok && n_cta < n_tiles) {
        __syncthreads();  // every thread is done with the staging buffer
        warp_tiles<MODE, IPT>(P, S, out, smem_raw, n_cta, n_tiles, tc);
    }
    finish_call(S, out, true);
}

// Two staging buffers: while a chunk is scored, the next one (of the same tile,
// or the first chunk of the CTA's next tile) is already on its way.  Tiles are
// claimed from the counter one tile ahead: while tile k is scored the CTA
// already knows tile k + 1 (its first chunk is staged during tile k) and the
// claim of tile k + 2 is in flight.
template <int MODE, int IPT, bool WARP>
__device__ __forceinline__ void score_body_pipe(const DevProblem &P, const BucketScratch &S,
                                                llama_decision *out, int32_t chunk, int32_t dl_cap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const size_t tbl = align16((size_t)chunk * (MODE == LLAMA_MODE_ALPHA ? 6 : 4));
    const size_t stage = tbl + 4 * (size_t)dl_cap;  // dl_cap is a multiple of 4
    uint16_t *c_s = reinterpret_cast<uint16_t *>(smem_raw + 2 * stage);
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ uint32_t red[IPT][kScoreThreads / 32];
    __shared__ long long next_tile;
    __shared__ TileConst tc;
    const int tid = threadIdx.x, H = P.n_hw;
    const uint32_t bar0 = smem_addr(&mbar[0]);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto lr_of = [&](int st) { return reinterpret_cast<uint16_t *>(smem_raw + st * stage); };
    auto dl_of = [&](int st) { return reinterpret_cast<int32_t *>(smem_raw + st * stage + tbl); };
    auto issue = [&](int st, const int4 &tx, int32_t c0) {
        // tx = {npad, dn, p0}
        const int32_t cn = min(chunk, tx.x - c0);
        uint16_t *lr = lr_of(st);
        stage_chunk<MODE>(P, (int64_t)tx.z, c0, cn, c0 == 0 && tx.y <= dl_cap, tx.y, lr, lr + chunk,
                          lr + 2 * chunk, dl_of(st), bar0 + 8 * st);
    };
    uint32_t phases = 0;   // bit st: parity of stage st's next completion
    uint32_t pending = 0;  // bit st: a copy into stage st is in flight
    bool ok = true;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    clear_counters(P, S);
    if (tid < H) tc.q[tid] = P.q[tid];
    // after a bucketing barrier gave up, no tile list or bucket entry is read
    const long long n_tiles = call_timed_out(S) ? 0 : (long long)S.ctrl[kCtrlTiles];
    // the whole-CTA tiles come first; the warp tiles after them (a kernel
    // without the warp phase scores any warp tile as a CTA tile of one lane
    // per invocation, with the same result)
    const long long n_cta =
        WARP && P.n_cta_ops < P.n_ops ? min((long long)S.ctrl[kCtrlCtaTiles], n_tiles) : n_tiles;
    long long ti = blockIdx.x, tn;
    if (tid == 0) next_tile = (long long)atomicAdd(&S.ctrl[kCtrlNextTile], 1ull) + gridDim.x;
    if (ti < n_cta) {
        if (tid == 0) issue(0, S.tiles[2 * ti + 1], 0);
        pending = 1u;
    }
    __syncthreads();
    tn = next_tile;
    int st = 0;
    TileState<IPT> T;
    while (ti < n_cta) {
        unsigned long long claim = 0;
        if (tid == 0) claim = atomicAdd(&S.ctrl[kCtrlNextTile], 1ull);  // the tile after tn
        const int4 txn = tn < n_cta ? S.tiles[2 * tn + 1] : make_int4(0, 0, 0, 0);
        tile_begin(P, S, ti, tc, T);
        const bool dl_staged = T.dn <= dl_cap;
        uint16_t *cg = c_s + T.g * IPT * H;
        for (int32_t c0 = 0; c0 < T.npad; c0 += chunk) {
            const int32_t cn = min(chunk, T.npad - c0);
            __syncthreads();  // every thread is done with the other stage and with cg
            // the item after this one: the next chunk, or the next tile's first
            if (c0 + chunk < T.npad || tn < n_cta) {
                if (tid == 0) {
                    if (c0 + chunk < T.npad) issue(st ^ 1, make_int4(T.npad, T.dn, (int32_t)T.p0, 0), c0 + chunk);
                    else issue(st ^ 1, txn, 0);
                }
                pending |= 1u << (st ^ 1);
            }
            if (c0 == 0 && !dl_staged) {
                if (S.b_cnt) counts_from_pass(S, T, H, c_s);
                else counts_from_global(P, S, T, tc, H, P.dlat + T.p0, cg);
            }
            if (!__syncthreads_and(mbar_wait(bar0 + 8 * st, (phases >> st) & 1u))) {
                ok = false;
                break;
            }
            phases ^= 1u << st;
            pending &= ~(1u << st);
            uint16_t *lr = lr_of(st);
            if (c0 == 0 && dl_staged) {
                counts_from_shared(S, T, tc, H, dl_of(st), cg);
                __syncthreads();
            }
            scan_chunk<MODE, IPT>(P, T, c0, cn, lr, lr + chunk, lr + 2 * chunk, cg);
            st ^= 1;
        }
        if (!ok) break;
        finish_tile<MODE, IPT>(P, S, out, T, tc, red);
        if (tid == 0) next_tile = (long long)(claim + gridDim.x);
        __syncthreads();
        ti = tn;
        tn = next_tile;
    }
    if (!ok) {
        // report, then wait (bounded) for every copy still in flight
        if (tid == 0) atomicOr(&S.ctrl[kCtrlTimeout], 1ull);
        for (int k = 0; k < 2; ++k)
            if (pending & (1u << k)) mbar_wait(bar0 + 8 * k, (phases >> k) & 1u);
    }
    if (WARP && ok && n_cta < n_tiles) {
        __syncthreads();  // every thread is done with the staging buffers
        warp_tiles<MODE, IPT>(P, S, out, smem_raw, n_cta, n_tiles, tc);
    }
    finish_call(S, out, true);
}

// Every (objective mode, invocations per thread, staging buffers) twice: with
// the warp phase (suffix w, for profiles with ops scored by warp tiles) and
// without it (fewer registers: more CTAs per SM where no op needs it).
#define LLAMA_SCORE_KERNEL(name, MODE, IPT, BODY, WARP)                                         \
    __global__ void __launch_bounds__(kScoreThreads)                                            \
        name(DevProblem P, BucketScratch S, llama_decision *out, int32_t chunk, int32_t dl_cap) { \
        BODY<MODE, IPT, WARP>(P, S, out, chunk, dl_cap);                                          \
    }
#define LLAMA_SCORE_KERNELS(name, MODE, IPT, BODY)  \
    LLAMA_SCORE_KERNEL(name, MODE, IPT, BODY, false) \
    LLAMA_SCORE_KERNEL(name##w, MODE, IPT, BODY, true)
LLAMA_SCORE_KERNELS(k_score_cf1, LLAMA_MODE_COST_FIRST, 1, score_body)
LLAMA_SCORE_KERNELS(k_score_cf2, LLAMA_MODE_COST_FIRST, 2, score_body)
LLAMA_SCORE_KERNELS(k_score_cf4, LLAMA_MODE_COST_FIRST, 4, score_body)
LLAMA_SCORE_KERNELS(k_score_al1, LLAMA_MODE_ALPHA, 1, score_body)
LLAMA_SCORE_KERNELS(k_score_al2, LLAMA_MODE_ALPHA, 2, score_body)
LLAMA_SCORE_KERNELS(k_score_al4, LLAMA_MODE_ALPHA, 4, score_body)
LLAMA_SCORE_KERNELS(k_score2_cf1, LLAMA_MODE_COST_FIRST, 1, score_body_pipe)
LLAMA_SCORE_KERNELS(k_score2_cf2, LLAMA_MODE_COST_FIRST, 2, score_body_pipe)
LLAMA_SCORE_KERNELS(k_score2_cf4, LLAMA_MODE_COST_FIRST, 4, score_body_pipe)
LLAMA_SCORE_KERNELS(k_score2_al1, LLAMA_MODE_ALPHA, 1, score_body_pipe)
LLAMA_SCORE_KERNELS(k_score2_al2, LLAMA_MODE_ALPHA, 2, score_body_pipe)
LLAMA_SCORE_KERNELS(k_score2_al4, LLAMA_MODE_ALPHA, 4, score_body_pipe)
#undef LLAMA_SCORE_KERNELS
#undef LLAMA_SCORE_KERNEL

const void *score_kernel(int mode, int ipt, int stages, bool warp) {
    // [warp][alpha][two stages][log2 ipt]
    static const void *const fn[2][2][2][3] = {
        {{{(const void *)k_score_cf1, (const void *)k_score_cf2, (const void *)k_score_cf4},
          {(const void *)k_score2_cf1, (const void *)k_score2_cf2, (const void *)k_score2_cf4}},
         {{(const void *)k_score_al1, (const void *)k_score_al2, (const void *)k_score_al4},
          {(const void *)k_score2_al1, (const void *)k_score2_al2, (const void *)k_score2_al4}}},
        {{{(const void *)k_score_cf1w, (const void *)k_score_cf2w, (const void *)k_score_cf4w},
          {(const void *)k_score2_cf1w, (const void *)k_score2_cf2w, (const void *)k_score2_cf4w}},
         {{(const void *)k_score_al1w, (const void *)k_score_al2w, (const void *)k_score_al4w},
          {(const void *)k_score2_al1w, (const void *)k_score2_al2w, (const void *)k_score2_al4w}}}};
    return fn[warp ? 1 : 0][mode == LLAMA_MODE_ALPHA ? 1 : 0][stages >= 2 ? 1 : 0][ipt >= 4 ? 2 : ipt == 2 ? 1 : 0];
}

// ---------------------------------------------------------------------------
// Staircase method (an exact rearrangement of the argmin of Eq. 1)
// ---------------------------------------------------------------------------

// Critical paths of every DAG (a1) for the staircase method: small DAGs one per
// warp, larger ones one per block.
__global__ void __launch_bounds__(256) k_critical_paths(DevProblem P, const int32_t *topo,
                                                        const int32_t *lvl_off, const int32_t *dag_lvl) {
    __shared__ CpSmem sm;
    critical_paths_of_block(P, blockIdx.x, gridDim.x, topo, lvl_off, dag_lvl, sm);
    asm volatile("griddepcontrol.launch_dependents;");
}

// One decision per thread.  For backend h the configurations of segment h that
// meet the slack are exactly those whose latency rank is below c_h, the number
// of the op's distinct latencies below slack(op, h); so the best key of the
// segment is stair[.. h ..][c_h], and the decision is the least of the H keys.
// c_h comes from the op's 32 first-round probe values (one line), then a
// bisection of the window they leave, all H searches in lockstep.
// For each backend h < n_hw <= MAXH, the count lo[h] of op g's distinct
// latencies below the invocation's slack floor(ref * (rbase - Q[h]) / cp) (0
// once the target has passed), one thread, every backend in lockstep: the op's
// 32 first-round probe values (one 128-byte line, probe l at ((l+1)*dn >> 5) -
// 1) leave, after c of them fall below the slack, the window [lo, hi] =
// [(c*dn >> 5), ((c+1)*dn >> 5) - 1].  With SECOND, a window of more than 32
// candidates is narrowed the same way by the 32 values of its second-round
// line (op, c).  A bisection closes what is left; each round issues every
// backend's loads before using any.
template <int MAXH, bool SECOND>
__device__ __forceinline__ void counts_all_backends(const DevProblem &P, int32_t g, int64_t ref, int64_t cp,
                                                    uint64_t mg, int64_t rbase, int32_t (&lo)[MAXH]) {
    const int H = P.n_hw;
    const int32_t dn = P.dlat_n[g];
    const int32_t *dl = P.dlat + P.pad_off[g];
    int32_t sl[MAXH], hi[MAXH];
#pragma unroll
    for (int h = 0; h < MAXH; ++h) {
        sl[h] = h < H ? slack_of(ref, cp, mg, rbase - P.q[h]) : 0;
        lo[h] = 0;
        hi[h] = h < H ? dn : 0;
    }
    if (dn > 32) {
        const int4 *pv = reinterpret_cast<const int4 *>(P.dpiv + 32 * (int64_t)g);
        int32_t cnt[MAXH];
#pragma unroll
        for (int h = 0; h < MAXH; ++h) cnt[h] = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const int4 q4 = __ldg(pv + w);
#pragma unroll
            for (int h = 0; h < MAXH; ++h)
                cnt[h] += (q4.x < sl[h]) + (q4.y < sl[h]) + (q4.z < sl[h]) + (q4.w < sl[h]);
        }
#pragma unroll
        for (int h = 0; h < MAXH; ++h) {
            if (h >= H) continue;
            const int32_t c = cnt[h];
            lo[h] = (c * dn) >> 5;
            hi[h] = c < 32 ? (((c + 1) * dn) >> 5) - 1 : dn;
        }
        if (SECOND && P.dpiv2 && dn > 32 * 33) {  // only then can a window exceed 32
            const int4 *lines[MAXH];
#pragma unroll
            for (int h = 0; h < MAXH; ++h) {
                lines[h] = reinterpret_cast<const int4 *>(P.dpiv2 + ((32 * (int64_t)g + cnt[h]) << 5));
                cnt[h] = 0;
            }
#pragma unroll
            for (int w = 0; w < 8; ++w) {
#pragma unroll
                for (int h = 0; h < MAXH; ++h) {
                    if (h >= H || hi[h] - lo[h] <= 32) continue;
                    const int4 q4 = __ldg(lines[h] + w);
                    cnt[h] += (q4.x < sl[h]) + (q4.y < sl[h]) + (q4.z < sl[h]) + (q4.w < sl[h]);
                }
            }
#pragma unroll
            for (int h = 0; h < MAXH; ++h) {
                const int32_t n = hi[h] - lo[h], c = cnt[h];
                if (h >= H || n <= 32) continue;
                hi[h] = c < 32 ? lo[h] + (((c + 1) * n) >> 5) - 1 : hi[h];
                lo[h] += (c * n) >> 5;
            }
        }
    }
    for (;;) {
        int32_t val[MAXH];
        bool more = false;
#pragma unroll
        for (int h = 0; h < MAXH; ++h) {  // all loads first
            const bool a = lo[h] < hi[h];
            more |= a;
            val[h] = a ? __ldg(dl + ((lo[h] + hi[h]) >> 1)) : 0;
        }
        if (!more) break;
#pragma unroll
        for (int h = 0; h < MAXH; ++h) {
            if (lo[h] >= hi[h]) continue;
            const int32_t mid = (lo[h] + hi[h]) >> 1;
            if (val[h] < sl[h]) lo[h] = mid + 1; else hi[h] = mid;
        }
    }
}

// The count pass of the scan method, between bucketing and scoring, for the
// ops whose distinct latencies the scoring kernel does not stage (more than
// dl_cap): one thread per bucket position computes the counts of every backend
// (counts_all_backends) into b_cnt, so the scoring kernel reads them instead of
// running a 32-lane search per (invocation, backend) -- a thread's search
// issues a few instructions per step where a warp-wide one issues a few
// hundred per search.  Only ops among the first n_big_ops of the bucket order
// can need counts, so only the positions before the first bucket of the
// others are visited.
template <int MAXH>
__global__ void __launch_bounds__(256, 4) k_counts(DevProblem P, BucketScratch S, int32_t dl_cap) {
    // the bucket entries and starts and the critical paths are visible after this
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int H = P.n_hw;
    // after a bucketing barrier gave up, the bucket starts and entries are not
    // this call's: nothing is read
    const int64_t n_pos = call_timed_out(S)             ? 0
                          : P.n_big_ops < P.n_ops ? (int64_t)S.op_start[P.op_order[P.n_big_ops]]
                                                  : (int64_t)S.ctrl[kCtrlPositions];
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n_pos;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int2 e = S.b_ent[p];
        const int32_t bi = e.x;
        if (!LLAMA_IN_BOUNDS(P, bi >= 0 && bi < S.n_inv, LLAMA_CHECK_COUNTS)) continue;
        const int32_t g = S.gop[bi];
        if (!LLAMA_IN_BOUNDS(P, g >= 0 && g < P.n_ops, LLAMA_CHECK_COUNTS)) continue;
        if (P.dlat_n[g] <= dl_cap) continue;
        int32_t lo[MAXH];
        counts_all_backends<MAXH, true>(P, g, P.ref[g], P.cp[g], P.cp_magic[g], (int64_t)e.y, lo);
#pragma unroll
        for (int h = 0; h < MAXH; ++h)
            if (h < H) S.b_cnt[p * H + h] = (uint16_t)lo[h];
    }
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
template __global__ void k_counts<4>(DevProblem, BucketScratch, int32_t);
template __global__ void k_counts<LLAMA_MAX_HW>(DevProblem, BucketScratch, int32_t);

// The staircase decision of one valid invocation of global op g whose
// remaining time before queueing is rbase = SLO - elapsed (Algorithm 1 with
// the queueing times P.q, Eq. 1 through the staircase tables): the decision,
// and its backend in *lam; with cnt_out, also the count per backend of the
// op's distinct latencies below the slack on it.
__device__ llama_decision stair_decide(const DevProblem &P, int32_t g, int64_t rbase, int *lam_out,
                                       int32_t *cnt_out = nullptr) {
    const int H = P.n_hw;
    const int64_t ref = P.ref[g], cp = P.cp[g];
    const uint64_t mg = P.cp_magic[g];
    int32_t lo[LLAMA_MAX_HW];
    counts_all_backends<LLAMA_MAX_HW, false>(P, g, ref, cp, mg, rbase, lo);
    if (cnt_out)
#pragma unroll
        for (int h = 0; h < LLAMA_MAX_HW; ++h) cnt_out[h] = lo[h];
    const uint16_t *sg = P.stair + P.stair_off[g];
    const int64_t stride = P.cfg_off[g + 1] - P.cfg_off[g] + 1;
    uint32_t key = 0xFFFFu;
#pragma unroll
    for (int h = 0; h < LLAMA_MAX_HW; ++h)
        if (h < H) key = min(key, (uint32_t)__ldg(sg + (int64_t)h * stride + lo[h]));
    const int64_t cb = P.cfg_off[g];
    if (!LLAMA_IN_BOUNDS(P, decode_key_ok(P, g, key, P.mode), LLAMA_CHECK_DECODE))
        key = P.mode == LLAMA_MODE_ALPHA ? 0u : 0xFFFFu;  // a key in bounds (the decision is then wrong)
    int4 dd;
    if (P.mode == LLAMA_MODE_ALPHA) dd = P.dec[2 * cb + key];
    else dd = key != 0xFFFFu ? P.dec[cb + key] : P.dfast[g];
    const int lam = dd.x >> 16;
    const int32_t slam = slack_of(ref, cp, mg, rbase - P.q[lam]);
    llama_decision dsn;
    dsn.cfg = dd.x & 0xFFFF;
    dsn.lat = dd.y;
    dsn.cost = (int64_t)(((uint64_t)(uint32_t)dd.w << 32) | (uint32_t)dd.z);
    dsn.slack = slam;
    dsn.flags = dd.y < slam ? LLAMA_FLAG_FEASIBLE : 0;
    if (lam_out) *lam_out = lam;
    return dsn;
}

__global__ void __launch_bounds__(256) k_stair(DevProblem P, int64_t n_inv, const int32_t *dag,
                                               const int32_t *op_local, const int64_t *start,
                                               int64_t now, BucketScratch S, llama_decision *out) {
    // the critical paths (previous kernel) are visible after this
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n_inv) {
        int32_t g;
        int64_t rbase;
        if (!invocation_op(P, dag[i], op_local[i], start[i], now, g, rbase)) {
            llama_decision bad;
            bad.cfg = -1;
            bad.lat = 0;
            bad.cost = 0;
            bad.slack = 0;
            bad.flags = LLAMA_FLAG_INVALID;
            out[i] = bad;
            atomicAdd(&S.ctrl[kCtrlInvalid], 1ull);
        } else {
            out[i] = stair_decide(P, g, rbase, nullptr);
        }
    }
    finish_call(S, out, false);
}

// ---------------------------------------------------------------------------
// Small calls of the scan method: no bucketing
// ---------------------------------------------------------------------------

// A warp per invocation (warp-uniform loop).  The decision is the one the
// bucketed scan reaches: the slack of each backend (Algorithm 1 from the
// critical paths of the previous kernel) becomes the count of the op's
// distinct latencies below it; every lane scans its share of the op's
// rank-encoded table, each vector against the count of its backend segment
// (Eq. 1's feasibility and objective in rank form, read from L2, where a call
// of few invocations leaves no table to share); a warp minimum of the packed
// keys; lane 0 decodes the least key.
//
// The counts: the searches of all backends advance together (their loads in
// flight at once).  While more than 32 candidates are left, each lane probes
// the last value of one of 32 equal blocks of them: the blocks whose last
// value is below the slack (a prefix, the values ascending) are wholly below
// it, and the first other block holds the boundary; then one probe per
// remaining candidate.  At most four rounds of loads for 32^3 distinct
// latencies.  The scan: four vectors per lane in flight.
template <int MODE>
__device__ __forceinline__ void direct_body(const DevProblem &P, int64_t n_inv, const int32_t *dag,
                                            const int32_t *op_local, const int64_t *start, int64_t now,
                                            const BucketScratch &S, llama_decision *out) {
    constexpr int kWarps = 256 / 32, kUnroll = 4;
    __shared__ TileConst tc;
    __shared__ uint32_t w_c2[kWarps][LLAMA_MAX_HW];  // per warp: count of each segment, both halves
    __shared__ int32_t w_end[kWarps][LLAMA_MAX_HW];  // per warp: end of each segment (vectors)
    const int H = P.n_hw, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // the critical paths (previous kernel) and the queueing times are visible after this
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if ((int)threadIdx.x < H) tc.q[threadIdx.x] = P.q[threadIdx.x];
    __syncthreads();
    const int64_t n_warps = (int64_t)gridDim.x * kWarps;
    for (int64_t i = blockIdx.x * (int64_t)kWarps + wid; i < n_inv; i += n_warps) {
        int32_t g;
        int64_t rbase;
        if (!invocation_op(P, dag[i], op_local[i], start[i], now, g, rbase)) {
            if (lane == 0) {
                llama_decision bad;
                bad.cfg = -1;
                bad.lat = 0;
                bad.cost = 0;
                bad.slack = 0;
                bad.flags = LLAMA_FLAG_INVALID;
                out[i] = bad;
                atomicAdd(&S.ctrl[kCtrlInvalid], 1ull);
            }
            continue;
        }
        // the remaining time before queueing, as a bucket entry holds it
        const int64_t rem = max(rbase, (int64_t)0);
        const int64_t ref = P.ref[g], cp = P.cp[g];
        const uint64_t mg = P.cp_magic[g];
        const int64_t p0 = P.pad_off[g];
        const int32_t dn = P.dlat_n[g];
        const int32_t *sp = P.seg_pad + (int64_t)g * (H + 1);
        const int32_t npad = __ldg(sp + H), beg = __ldg(sp) / kVec;
        if (!LLAMA_IN_BOUNDS(P, p0 >= 0 && p0 + npad <= P.n_pad && dn <= npad, LLAMA_CHECK_TILE)) continue;
        const int32_t *dl = P.dlat + p0;
        int32_t sl[LLAMA_MAX_HW], lo[LLAMA_MAX_HW], hi[LLAMA_MAX_HW];
#pragma unroll
        for (int h = 0; h < LLAMA_MAX_HW; ++h) {
            sl[h] = h < H ? slack_of(ref, cp, mg, rem - tc.q[h]) : 0;
            lo[h] = 0;
            hi[h] = h < H ? dn : 0;
        }
        for (;;) {  // each round leaves fewer than 1/32 of the candidates
            bool any = false, below[LLAMA_MAX_HW];
            int32_t step[LLAMA_MAX_HW];
#pragma unroll
            for (int h = 0; h < LLAMA_MAX_HW; ++h) {
                const bool act = hi[h] - lo[h] > 32;
                any |= act;
                step[h] = act ? (hi[h] - lo[h] + 31) / 32 : 0;
                const int32_t p = lo[h] + (lane + 1) * step[h] - 1;
                below[h] = act && p < hi[h] && __ldg(dl + p) < sl[h];
            }
            if (!any) break;
#pragma unroll
            for (int h = 0; h < LLAMA_MAX_HW; ++h) {
                if (step[h] == 0) continue;
                lo[h] += __popc(__ballot_sync(0xffffffffu, below[h])) * step[h];
                hi[h] = min(hi[h], lo[h] + step[h] - 1);  // the first block not below ends at a value >= s
            }
        }
        {
            bool below[LLAMA_MAX_HW];
#pragma unroll
            for (int h = 0; h < LLAMA_MAX_HW; ++h) below[h] = lo[h] + lane < hi[h] && __ldg(dl + lo[h] + lane) < sl[h];
#pragma unroll
            for (int h = 0; h < LLAMA_MAX_HW; ++h) {
                const int32_t c = lo[h] + __popc(__ballot_sync(0xffffffffu, below[h]));
                if (lane == h && h < H) {
                    w_c2[wid][h] = (uint32_t)c * 0x00010001u;
                    w_end[wid][h] = __ldg(sp + h + 1) / kVec;
                }
            }
        }
        __syncwarp();
        const uint4 *lr4 = reinterpret_cast<const uint4 *>(P.lrb + p0);
        const uint4 *rf4 = reinterpret_cast<const uint4 *>(P.rf + p0);
        const uint4 *df4 = reinterpret_cast<const uint4 *>(P.df + p0);
        const int nv = npad / kVec;
        uint32_t best = 0xFFFFFFFFu;
        int h = 0;  // the segment of this lane's vector (non-decreasing along the loop)
        for (int q0 = beg + lane; q0 < nv; q0 += 32 * kUnroll) {
            uint4 lk[kUnroll], rk[kUnroll], dk[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const int q = q0 + 32 * u;
                if (q < nv) {
                    lk[u] = __ldg(lr4 + q);
                    rk[u] = __ldg(rf4 + q);
                    if (MODE == LLAMA_MODE_ALPHA) dk[u] = __ldg(df4 + q);
                }
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const int q = q0 + 32 * u;
                if (q >= nv) break;
                while (q >= w_end[wid][h]) ++h;  // the last segment ends at nv
                if (MODE == LLAMA_MODE_ALPHA) best = scan8_alpha(best, w_c2[wid][h], lk[u], rk[u], dk[u]);
                else best = scan8_cost_first(best, w_c2[wid][h], lk[u], rk[u]);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = vmin_u16x2(best, __shfl_xor_sync(0xffffffffu, best, o));
        if (lane == 0)
            decode_into<MODE>(P, g, (int32_t)P.cfg_off[g], min(best & 0xFFFFu, best >> 16), ref, cp, mg, rem, tc,
                              out + i);
        __syncwarp();  // the warp's segment words are read before the next invocation writes them
    }
    finish_call(S, out, false);
}

__global__ void __launch_bounds__(256) k_direct_cf(DevProblem P, int64_t n_inv, const int32_t *dag,
                                                   const int32_t *op_local, const int64_t *start, int64_t now,
                                                   BucketScratch S, llama_decision *out) {
    direct_body<LLAMA_MODE_COST_FIRST>(P, n_inv, dag, op_local, start, now, S, out);
}

__global__ void __launch_bounds__(256) k_direct_al(DevProblem P, int64_t n_inv, const int32_t *dag,
                                                   const int32_t *op_local, const int64_t *start, int64_t now,
                                                   BucketScratch S, llama_decision *out) {
    direct_body<LLAMA_MODE_ALPHA>(P, n_inv, dag, op_local, start, now, S, out);
}

// Inclusive minimum scan of a[0..n) in shared memory by the whole block, from
// the front (reverse = false) or from the back; part[] holds 32 words.
template <typename T>
__device__ void block_min_scan(T *a, int n, bool reverse, T *part) {
    const T kTop = sizeof(T) == 8 ? (T)LLONG_MAX : (T)INT32_MAX;  // int32_t or long long
    const int NT = blockDim.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int per = (n + NT - 1) / NT;
    const int b = min(n, tid * per), e = min(n, b + per);
    auto at = [&](int k) -> T & { return a[reverse ? n - 1 - k : k]; };
    T run = kTop;
    for (int k = b; k < e; ++k) run = min(run, at(k));
    T inc = run;
    for (int o = 1; o < 32; o <<= 1) {
        const T u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc = min(inc, u);
    }
    if (lane == 31) part[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        T w = lane < (NT >> 5) ? part[lane] : kTop;
        for (int o = 1; o < 32; o <<= 1) {
            const T u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w = min(w, u);
        }
        if (lane < (NT >> 5)) part[lane] = w;
    }
    __syncthreads();
    // minimum of everything before this thread's run
    T before = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) before = kTop;
    if (wid > 0) before = min(before, part[wid - 1]);
    for (int k = b; k < e; ++k) {
        before = min(before, at(k));
        at(k) = before;
    }
    __syncthreads();
}

// Staircase tables, one CTA per op: for each backend segment, the keys of its
// configurations at their latency ranks, then a prefix minimum (feasible
// branch: configurations below rank k) and, in alpha mode, a suffix minimum
// (infeasible branch: configurations at or above rank k).
__global__ void k_encode_stair(DevProblem P, uint16_t *stair) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int32_t part[32];
    const int v = blockIdx.x, H = P.n_hw, T = blockDim.x, tid = threadIdx.x;
    if (P.encode_only && !P.encode_only[v]) return;
    const bool alpha = P.mode == LLAMA_MODE_ALPHA;
    const int32_t dn = P.dlat_n[v], m = dn + 1;
    int32_t *pre = reinterpret_cast<int32_t *>(smem_raw);
    int32_t *suf = pre + m;
    const int64_t p0 = P.pad_off[v];
    const int32_t *hw = P.hw_off + (int64_t)v * (H + 1);
    const int32_t *sp = P.seg_pad + (int64_t)v * (H + 1);
    uint16_t *out = stair + P.stair_off[v];
    const int64_t stride = P.cfg_off[v + 1] - P.cfg_off[v] + 1;  // n_cfg(v) + 1 >= m
    for (int h = 0; h < H; ++h) {
        for (int k = tid; k < m; k += T) {
            pre[k] = 0xFFFF;
            suf[k] = 0xFFFF;
        }
        __syncthreads();
        const int n_h = hw[h + 1] - hw[h];
        for (int j = tid; j < n_h; j += T) {
            const int64_t pp = p0 + sp[h] + j;
            const int32_t r = (int32_t)P.lrb[pp] - kLatRankBias;
            const int32_t f = P.rf[pp];
            atomicMin(&pre[r + 1], f);
            if (alpha) atomicMin(&suf[r], f ^ (int32_t)P.df[pp]);
        }
        __syncthreads();
        block_min_scan(pre, m, false, part);
        if (alpha) block_min_scan(suf, m, true, part);
        for (int k = tid; k < m; k += T)
            out[(int64_t)h * stride + k] = (uint16_t)(alpha ? min(pre[k], suf[k]) : pre[k]);
        __syncthreads();
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

// Eq. 3's per-backend minima as tables, one CTA per op (used where the
// minima of single invocations are needed fast: the serving loop's commit).
// For segment h and a count k of the op's distinct latencies below the
// slack on h, a configuration of h is feasible exactly when its latency rank
// is below k, so the least Eq. 1 objective on h is
//   min(least C among ranks < k, least C + floor(a L R / (b B R_total)) among ranks >= k),
// a prefix minimum and a suffix minimum over the ranks; at
// objmin[stair_off[v] + h*(n_cfg(v)+1) + k] for k = 0..dn (INT64_MAX for an
// empty segment), the staircase tables' indexing.
__global__ void k_encode_objmin(DevProblem P, int64_t *objmin) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ long long part[32];
    const int v = blockIdx.x, H = P.n_hw, T = blockDim.x, tid = threadIdx.x;
    const int32_t dn = P.dlat_n[v], m = dn + 1;
    long long *pre = reinterpret_cast<long long *>(smem_raw);
    long long *suf = pre + m;
    const int64_t p0 = P.pad_off[v], c0 = P.cfg_off[v];
    const int32_t *hw = P.hw_off + (int64_t)v * (H + 1);
    const int32_t *sp = P.seg_pad + (int64_t)v * (H + 1);
    int64_t *out = objmin + P.stair_off[v];
    const int64_t stride = P.cfg_off[v + 1] - c0 + 1;
    for (int h = 0; h < H; ++h) {
        for (int k = tid; k < m; k += T) {
            pre[k] = LLONG_MAX;
            suf[k] = LLONG_MAX;
        }
        __syncthreads();
        const int n_h = hw[h + 1] - hw[h];
        for (int j = tid; j < n_h; j += T) {
            const int32_t r = (int32_t)P.lrb[p0 + sp[h] + j] - kLatRankBias;
            const int64_t g = c0 + hw[h] + j;
            atomicMin(&pre[r + 1], (long long)P.cost[g]);
            atomicMin(&suf[r], (long long)alpha_infeasible_objective(P, g, h));
        }
        __syncthreads();
        block_min_scan(pre, m, false, part);
        block_min_scan(suf, m, true, part);
        for (int k = tid; k < m; k += T) out[(int64_t)h * stride + k] = min(pre[k], suf[k]);
        __syncthreads();
    }
}

cudaError_t enqueue_encode_objmin(const ContextView &v, int64_t *objmin, cudaStream_t s) {
    // distinct latencies of an op <= its configurations
    const size_t smem = 2 * sizeof(long long) * (size_t)(v.max_ncfg + 1);
    cudaError_t e = cudaFuncSetAttribute(k_encode_objmin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (v.n_ops > 0) k_encode_objmin<<<v.n_ops, 1024, smem, s>>>(v.P, objmin);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The launch sequence of one scheduling call
// ---------------------------------------------------------------------------

int64_t max_tiles(int64_t n_inv, int32_t n_ops) { return n_inv + n_ops; }

int schedule_launches(const ContextView &v, const BucketScratch &S, int64_t n_inv) {
    if (v.method == LLAMA_METHOD_STAIRCASE || n_inv <= v.direct_max) return 2;
    return S.b_cnt && v.need_counts ? 3 : 2;
}

// After a failed launch that followed a successful one: the kernels already
// enqueued may have counted invocations, so the per-op counters and the
// control and status words are cleared on the same stream (memsets, nothing
// allocated) and the scratch is ready for the next call.
static cudaError_t clear_scratch_after_error(const ContextView &v, const BucketScratch &S, cudaStream_t s,
                                             cudaError_t err) {
    cudaGetLastError();  // the launch error itself is not sticky
    cudaMemsetAsync(S.cnt, 0, sizeof(int32_t) * kCntStride * (size_t)v.n_ops, s);
    cudaMemsetAsync(S.ctrl, 0, sizeof(unsigned long long) * (kCtrlWords + kStatusWords), s);
    return err;
}

static cudaError_t enqueue_schedule_impl(const ContextView &v, const BucketScratch &S, int64_t n_inv,
                                         const int32_t *dag, const int32_t *op_local, const int64_t *start,
                                         int64_t now, llama_decision *out, cudaStream_t s,
                                         const cudaEvent_t *trace, bool &launched);

cudaError_t enqueue_schedule(const ContextView &v, const BucketScratch &S0, int64_t n_inv,
                             const int32_t *dag, const int32_t *op_local, const int64_t *start,
                             int64_t now, llama_decision *out, cudaStream_t s,
                             const cudaEvent_t *trace) {
    BucketScratch S = S0;
    S.n_inv = n_inv;
    bool launched = false;
    const cudaError_t e = enqueue_schedule_impl(v, S, n_inv, dag, op_local, start, now, out, s, trace, launched);
    if (e != cudaSuccess && launched) return clear_scratch_after_error(v, S, s, e);
    return e;
}

static cudaError_t enqueue_schedule_impl(const ContextView &v, const BucketScratch &S, int64_t n_inv,
                                         const int32_t *dag, const int32_t *op_local, const int64_t *start,
                                         int64_t now, llama_decision *out, cudaStream_t s,
                                         const cudaEvent_t *trace, bool &launched) {
    auto mark = [&](int k) { if (trace) cudaEventRecord(trace[k], s); };
    mark(0);
    cudaError_t e = cudaSuccess;
    if (v.method == LLAMA_METHOD_STAIRCASE) {
        k_critical_paths<<<std::max(1, (v.n_dags + 7) / 8), 256, 0, s>>>(v.P, v.topo, v.lvl_off, v.dag_lvl);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        launched = true;
        mark(1);
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)((n_inv + 255) / 256));
        cfg.blockDim = dim3(256);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = trace ? 0 : 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        DevProblem P = v.P;
        BucketScratch Sc = S;
        void *args[] = {&P, &n_inv, &dag, &op_local, &start, &now, &Sc, &out};
        e = cudaLaunchKernelExC(&cfg, (const void *)k_stair, args);
        if (e != cudaSuccess) return e;
        mark(2);
        return cudaGetLastError();
    }
    if (n_inv <= v.direct_max) {
        // a small call: critical paths, then a warp per invocation
        k_critical_paths<<<std::max(1, (v.n_dags + 7) / 8), 256, 0, s>>>(v.P, v.topo, v.lvl_off, v.dag_lvl);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        launched = true;
        mark(1);
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)std::max<int64_t>(1, (n_inv + 7) / 8));
        cfg.blockDim = dim3(256);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = trace ? 0 : 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        DevProblem P = v.P;
        BucketScratch Sc = S;
        void *args[] = {&P, &n_inv, &dag, &op_local, &start, &now, &Sc, &out};
        e = cudaLaunchKernelExC(&cfg, v.mode == LLAMA_MODE_ALPHA ? (const void *)k_direct_al : (const void *)k_direct_cf,
                                args);
        if (e != cudaSuccess) return e;
        mark(2);
        return cudaGetLastError();
    }
    // bucketing: one cooperative launch (its blocks meet at a grid barrier)
    const int n_cp = std::max(1, std::min((v.n_dags + 7) / 8, std::max(1, v.bucket_max_blocks / 4)));
    // counting blocks: enough for the invocations, and for the bucket layout
    // (one run of ops per block) enough that no block lays out more than 256 ops
    const int count_blocks = (int)std::max<int64_t>(
        1, std::min<int64_t>(std::max<int64_t>((n_inv + 255) / 256, (v.n_ops + 255) / 256),
                             (int64_t)v.bucket_max_blocks - n_cp));
    {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(n_cp + count_blocks);
        cfg.blockDim = dim3(256);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        DevProblem P = v.P;
        BucketScratch Sc = S;
        const int32_t *topo = v.topo, *lvl_off = v.lvl_off, *dag_lvl = v.dag_lvl;
        int32_t min_vpl = v.min_vpl, ipt = v.ipt, ncp = n_cp;
        void *args[] = {&P, &n_inv, &dag, &op_local, &start, &now, &Sc, &out,
                        &topo, &lvl_off, &dag_lvl, &min_vpl, &ipt, &ncp};
        e = cudaLaunchKernelExC(&cfg, (const void *)k_bucket, args);
        if (e != cudaSuccess) return e;
        launched = true;
    }
    mark(1);
    // the count pass, where some op's distinct latencies are not staged by the
    // scoring kernel (and the scratch has room for the counts); the scoring
    // kernel reads the counts only when it ran
    BucketScratch Sc = S;
    if (S.b_cnt && v.need_counts) {
        cudaLaunchConfig_t cfg{};
        // a thread per bucket position, at most four resident blocks per SM (the
        // threads stride over the positions, whose number only the device knows)
        cfg.gridDim = dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>((n_inv + 255) / 256,
                                                                            (int64_t)v.num_sms * 4)));
        cfg.blockDim = dim3(256);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = trace ? 0 : 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        DevProblem P = v.P;
        int32_t dl_cap = v.dlat_cap;
        void *args[] = {&P, &Sc, &dl_cap};
        e = cudaLaunchKernelExC(&cfg, v.n_hw <= 4 ? (const void *)k_counts<4> : (const void *)k_counts<LLAMA_MAX_HW>,
                                args);
        if (e != cudaSuccess) return e;
    } else {
        Sc.b_cnt = nullptr;
    }
    // the scoring kernel may launch before the previous kernel completes (it
    // waits on griddepcontrol.wait before reading the bucketing output)
    cudaLaunchConfig_t cfg{};
    // a call has at most n_inv tiles: a small call leaves the rest of the GPU
    // to calls running beside it
    cfg.gridDim = dim3((unsigned)std::min<int64_t>(v.score_grid, std::max<int64_t>(1, n_inv)));
    cfg.blockDim = dim3(kScoreThreads);
    cfg.dynamicSmemBytes = v.score_smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = trace ? 0 : 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    DevProblem P = v.P;
    int32_t chunk = v.score_chunk, dl_cap = v.dlat_cap;
    void *args[] = {&P, &Sc, &out, &chunk, &dl_cap};
    e = cudaLaunchKernelExC(&cfg, score_kernel(v.mode, v.ipt, v.stages, v.warp_tiles), args);
    if (e != cudaSuccess) return e;
    mark(2);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Encoding of the tables (llama_set_profiles)
// ---------------------------------------------------------------------------

// One CTA per op: latencies into the padded layout (INT32_MAX at pads, which no
// slack can exceed), ranks initialised to the pad rank, and the op's fastest
// configuration argmin (L, index).
// One CTA per op: pads get the pad ranks (never feasible, never the minimum),
// and the op's fastest configuration argmin (L, index) is recorded.
__global__ void k_encode_pad(DevProblem P, uint16_t *lrb, uint16_t *rf, uint16_t *df, int32_t *fast) {
    __shared__ int64_t red[32];
    const int v = blockIdx.x, H = P.n_hw;
    if (P.encode_only && !P.encode_only[v]) return;
    const int64_t c0 = P.cfg_off[v], p0 = P.pad_off[v];
    const int32_t *hw = P.hw_off + (int64_t)v * (H + 1);
    const int32_t *sp = P.seg_pad + (int64_t)v * (H + 1);
    for (int h = 0; h < H; ++h) {
        const int src_n = hw[h + 1] - hw[h], dst_n = sp[h + 1] - sp[h];
        for (int k = threadIdx.x; k < dst_n; k += blockDim.x) {
            const int64_t dst = p0 + sp[h] + k;
            if (k >= src_n) lrb[dst] = kLatRankPad;
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

// One CTA per op: sort the op's (objective, tag) pairs in shared memory with a
// bitonic network and write the ranks.  COST_FIRST sorts (C/B, x); ALPHA sorts
// the 2n values {(C/B, 2x), (infeasible objective, 2x+1)} jointly.
__global__ void k_encode_rank(DevProblem P, int32_t sort_cap, uint16_t *rf, uint16_t *df,
                              uint16_t *inv) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *key = reinterpret_cast<uint64_t *>(smem_raw);
    uint32_t *tag = reinterpret_cast<uint32_t *>(smem_raw + 8 * (size_t)sort_cap);
    const int v = blockIdx.x, H = P.n_hw, T = blockDim.x;
    if (P.encode_only && !P.encode_only[v]) return;
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

// One CTA per op: sort the op's (latency, index) pairs in shared memory
// (bitonic network), keep the distinct latencies in ascending order
// (dlat[pad_off[v] ..], dlat_n[v] of them) and write each configuration's
// biased latency rank 0x8000 + (position of its latency among the distinct
// ones) at its padded position.
__global__ void k_encode_lat(DevProblem P, uint16_t *lrb, int32_t *dlat, int32_t *dlat_n) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *key = reinterpret_cast<uint64_t *>(smem_raw);
    __shared__ int32_t warp_tot[32];
    const int v = blockIdx.x, H = P.n_hw, T = blockDim.x, tid = threadIdx.x;
    if (P.encode_only && !P.encode_only[v]) return;
    const int lane = tid & 31, wid = tid >> 5;
    const int64_t c0 = P.cfg_off[v], p0 = P.pad_off[v];
    const int n = (int)(P.cfg_off[v + 1] - c0);
    int N = 1;
    while (N < n) N <<= 1;
    const int32_t *hw = P.hw_off + (int64_t)v * (H + 1);
    const int32_t *sp = P.seg_pad + (int64_t)v * (H + 1);
    for (int k = tid; k < N; k += T)
        key[k] = k < n ? ((uint64_t)(uint32_t)P.lat[c0 + k] << 16) | (uint64_t)k : ~0ull;
    __syncthreads();
    for (int kk = 2; kk <= N; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < N; i += T) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & kk) == 0;
                    if ((key[i] > key[ixj]) == up) {
                        const uint64_t t = key[i];
                        key[i] = key[ixj];
                        key[ixj] = t;
                    }
                }
            }
            __syncthreads();
        }
    }
    // rank of sorted entry r = (number of distinct latencies among entries 0..r) - 1:
    // an inclusive block scan of "differs from its predecessor" flags, in
    // contiguous runs of `per` entries per thread
    const int per = (n + T - 1) / T;
    const int b = min(n, tid * per), e = min(n, b + per);
    int32_t cnt = 0;
    for (int r = b; r < e; ++r) cnt += (r == 0 || (key[r] >> 16) != (key[r - 1] >> 16)) ? 1 : 0;
    int32_t inc = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int32_t w = lane < (T >> 5) ? warp_tot[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += u;
        }
        if (lane < (T >> 5)) warp_tot[lane] = w;
    }
    __syncthreads();
    int32_t rank = inc - cnt + (wid > 0 ? warp_tot[wid - 1] : 0) - 1;
    for (int r = b; r < e; ++r) {
        const int32_t L = (int32_t)(key[r] >> 16);
        if (r == 0 || L != (int32_t)(key[r - 1] >> 16)) {
            ++rank;
            dlat[p0 + rank] = L;
        }
        const int x = (int)(key[r] & 0xFFFF);
        const int lam = backend_of(hw, H, x);
        lrb[p0 + sp[lam] + (x - hw[lam])] = (uint16_t)(kLatRankBias + rank);
    }
    if (tid == T - 1) dlat_n[v] = warp_tot[(T >> 5) - 1];
}

// The 32 first-round probe values of every op with more than 32 distinct
// latencies (one thread per value).
__global__ void k_encode_piv(DevProblem P, int32_t *dpiv) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= 32 * (int64_t)P.n_ops) return;
    const int32_t v = (int32_t)(k >> 5), l = (int32_t)(k & 31), dn = P.dlat_n[v];
    if (P.encode_only && !P.encode_only[v]) return;
    dpiv[k] = dn > 32 ? P.dlat[P.pad_off[v] + (((l + 1) * dn) >> 5) - 1] : INT32_MAX;
}

// Second-round probe lines: one 128-byte line per (op, outcome c of the first
// round), so a search's second round reads one line instead of bisecting the
// window the first round leaves.  Lines of windows of 32 or fewer candidates
// are unused.
__global__ void k_encode_piv2(DevProblem P, int32_t *dpiv2) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= 1024 * (int64_t)P.n_ops) return;
    const int32_t v = (int32_t)(k >> 10), c = (int32_t)((k >> 5) & 31), l = (int32_t)(k & 31);
    if (P.encode_only && !P.encode_only[v]) return;
    const int32_t dn = P.dlat_n[v];
    const int32_t lo = (c * dn) >> 5, n = ((((c + 1) * dn) >> 5) - 1) - lo;
    dpiv2[k] = dn > 32 && n > 32 ? P.dlat[P.pad_off[v] + lo + (((l + 1) * n) >> 5) - 1] : INT32_MAX;
}

// Decode tables (one CTA per op): the configuration behind every rank, and the
// fastest one.
__global__ void k_encode_dec(DevProblem P, int4 *dec, int4 *dfast) {
    const int v = blockIdx.x, H = P.n_hw;
    if (P.encode_only && !P.encode_only[v]) return;
    const int64_t c0 = P.cfg_off[v];
    const int n = (int)(P.cfg_off[v + 1] - c0);
    const bool alpha = P.mode == LLAMA_MODE_ALPHA;
    const int cnt = alpha ? 2 * n : n;
    const int64_t off = alpha ? 2 * c0 : c0;
    const int32_t *hw = P.hw_off + (int64_t)v * (H + 1);
    auto entry = [&](int x) {
        const int64_t g = c0 + x;
        const uint64_t cost = (uint64_t)P.cost[g];
        return make_int4(x | (backend_of(hw, H, x) << 16), P.lat[g], (int32_t)(uint32_t)cost,
                         (int32_t)(uint32_t)(cost >> 32));
    };
    for (int r = threadIdx.x; r < cnt; r += blockDim.x) dec[off + r] = entry(P.inv[2 * c0 + r]);
    if (threadIdx.x == 0) dfast[v] = entry(P.fast[v]);
}

// Eq. 2 over the decided invocations (valid ones): their latency times their
// requested resources, summed per backend.  A backend's sum saturates at
// cap(h) = INT32_MAX * R_total(h): every sum at or above it floors to a
// queueing time of at least INT32_MAX, which k_queue_finish clamps to
// INT32_MAX, so saturating keeps the result exact while no partial sum can
// wrap (each term is below 2^47, every saturated value below 2^62, so a sum
// of two never exceeds 2^63).
__device__ __forceinline__ unsigned long long queue_cap(const DevProblem &P, int h) {
    return (unsigned long long)INT32_MAX * (unsigned long long)(uint32_t)P.res_total[h];
}

__global__ void k_queue_sum(DevProblem P, int64_t n, const int32_t *dag, const int32_t *op_local,
                            const llama_decision *dec, unsigned long long *sums) {
    const int H = P.n_hw;
    unsigned long long loc[LLAMA_MAX_HW], cap[LLAMA_MAX_HW];
#pragma unroll
    for (int h = 0; h < LLAMA_MAX_HW; ++h) {
        loc[h] = 0;
        cap[h] = h < H ? queue_cap(P, h) : 0;
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const llama_decision d = dec[i];
        if (d.cfg < 0 || (d.flags & LLAMA_FLAG_INVALID)) continue;
        const int32_t dg = dag[i], o = op_local[i];
        if (dg < 0 || dg >= P.n_dags || o < 0 || o >= P.dag_op_off[dg + 1] - P.dag_op_off[dg]) continue;
        const int32_t v = P.dag_op_off[dg] + o;
        const int64_t g = P.cfg_off[v] + d.cfg;
        if (d.cfg >= P.cfg_off[v + 1] - P.cfg_off[v]) continue;
        const int lam = backend_of(P.hw_off + (int64_t)v * (H + 1), H, d.cfg);
        const unsigned long long w = (unsigned long long)(uint32_t)d.lat * (unsigned long long)(uint32_t)P.res[g];
#pragma unroll
        for (int h = 0; h < LLAMA_MAX_HW; ++h)
            if (h == lam) loc[h] = min(loc[h] + w, cap[h]);
    }
#pragma unroll
    for (int h = 0; h < LLAMA_MAX_HW; ++h) {
        unsigned long long v = loc[h];
        for (int o = 16; o > 0; o >>= 1) v = min(v + __shfl_xor_sync(0xffffffffu, v, o), cap[h]);
        if ((threadIdx.x & 31) == 0 && h < H && v) {
            // saturating atomic add: both operands are at most cap(h) < 2^62
            unsigned long long old = sums[h], seen;
            do {
                seen = old;
                old = atomicCAS(sums + h, seen, min(seen + v, cap[h]));
            } while (old != seen);
        }
    }
}

__global__ void k_queue_finish(DevProblem P, const unsigned long long *sums, int64_t *q_out, int64_t *q_ctx) {
    const int h = threadIdx.x;
    if (h >= P.n_hw) return;
    const unsigned long long q = sums[h] / (unsigned long long)P.res_total[h];
    const int64_t v = q > (unsigned long long)INT32_MAX ? (int64_t)INT32_MAX : (int64_t)q;
    if (q_out) q_out[h] = v;
    if (q_ctx) q_ctx[h] = v;
}

// Eq. 3 (Section 4.4): for invocation i and backend h, the least objective of
// Eq. 1 among op's configurations on h, each against slack(op, h): C/B if
// L < slack, else C/B + floor(alpha_num L R / (alpha_den B R_total)),
// saturating at INT64_MAX; INT64_MAX for an empty segment or an invalid
// invocation.  One warp per invocation.
// The least Eq. 1 objective per backend among the configurations of global op
// v, each against the slack of its own backend sl[lambda(x)], by the 32 lanes
// of a warp (configurations strided over the lanes, then a warp minimum):
// every lane returns the minima in best[] (INT64_MAX for an empty backend).
__device__ void warp_backend_minima(const DevProblem &P, int32_t v, const int32_t (&sl)[LLAMA_MAX_HW],
                                    int64_t (&best)[LLAMA_MAX_HW]) {
    const int H = P.n_hw, lane = threadIdx.x & 31;
#pragma unroll
    for (int h = 0; h < LLAMA_MAX_HW; ++h) best[h] = INT64_MAX;
    const int64_t c0 = P.cfg_off[v];
    const int n = (int)(P.cfg_off[v + 1] - c0);
    const int32_t *hw = P.hw_off + (int64_t)v * (H + 1);
    for (int x = lane; x < n; x += 32) {
        const int lam = backend_of(hw, H, x);
        const int64_t g = c0 + x;
        int32_t s = sl[0];
#pragma unroll
        for (int h = 1; h < LLAMA_MAX_HW; ++h)
            if (h == lam) s = sl[h];
        const int64_t obj = P.lat[g] < s ? P.cost[g] : (int64_t)alpha_infeasible_objective(P, g, lam);
#pragma unroll
        for (int h = 0; h < LLAMA_MAX_HW; ++h)
            if (h == lam) best[h] = min(best[h], obj);
    }
#pragma unroll
    for (int h = 0; h < LLAMA_MAX_HW; ++h)
        for (int k = 16; k > 0; k >>= 1)
            best[h] = min(best[h], (int64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)best[h], k));
}

// Eq. 3's affinity of a decision on backend lam given the per-backend minima:
// the least objective on the other backends over the least on lam, as doubles
// (objectives stay below 2^53: exact conversions); +inf when its own is 0,
// 1.0 when both are.
__device__ __forceinline__ double affinity_of(const int64_t *obj_min, int H, int lam) {
    int64_t other = INT64_MAX;
    for (int h = 0; h < H; ++h)
        if (h != lam) other = min(other, obj_min[h]);
    const int64_t own = obj_min[lam];
    return own == 0 ? (other == 0 ? 1.0 : INFINITY) : (double)other / (double)own;
}

__global__ void k_backend_obj(DevProblem P, int64_t n_inv, const int32_t *dag, const int32_t *op_local,
                              const int64_t *start, int64_t now, int64_t *obj_min) {
    const int H = P.n_hw, lane = threadIdx.x & 31;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= n_inv) return;
    int64_t best[LLAMA_MAX_HW];
#pragma unroll
    for (int h = 0; h < LLAMA_MAX_HW; ++h) best[h] = INT64_MAX;
    const int32_t d = dag[i], o = op_local[i];
    if (invocation_valid(P, d, o, start[i], now)) {
        const int32_t v = P.dag_op_off[d] + o;
        const int64_t rbase = P.slo[d] - (now - start[i]);
        int32_t sl[LLAMA_MAX_HW];
#pragma unroll
        for (int h = 0; h < LLAMA_MAX_HW; ++h)
            sl[h] = h < H ? slack_of(P.ref[v], P.cp[v], P.cp_magic[v], rbase - P.q[h]) : 0;
        warp_backend_minima(P, v, sl, best);
    }
    if (lane == 0)
        for (int h = 0; h < H; ++h) obj_min[i * H + h] = best[h];
}

// Priority-based commit (Section 4.4): the affinity of each decided
// invocation to the backend of its configuration, min over the other
// backends / min over its own (Eq. 3), and sort keys for the order (backend
// ascending, affinity descending, then index).
__global__ void k_commit_keys(DevProblem P, int64_t n, const int32_t *dag, const int32_t *op_local,
                              const llama_decision *dec, const int64_t *obj_min, uint64_t *aff_key,
                              uint32_t *lam_key, int32_t *idx, double *aff_out) {
    const int H = P.n_hw;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const llama_decision dd = dec[i];
        int lam = H;  // invalid decisions go last
        double aff = 0.0;
        if (dd.cfg >= 0 && !(dd.flags & LLAMA_FLAG_INVALID)) {
            const int32_t v = P.dag_op_off[dag[i]] + op_local[i];
            lam = backend_of(P.hw_off + (int64_t)v * (H + 1), H, dd.cfg);
            aff = affinity_of(obj_min + i * H, H, lam);
        }
        // descending affinity: invert the order-preserving bit pattern of a non-negative double
        aff_key[i] = ~(uint64_t)__double_as_longlong(aff);
        lam_key[i] = (uint32_t)lam;
        idx[i] = (int32_t)i;
        if (aff_out) aff_out[i] = aff;
    }
}

__global__ void k_gather_u32(int64_t n, const uint32_t *src, const int32_t *idx, uint32_t *dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[idx[i]];
}

// Feedback, step 1: validate the observations and key them by global
// configuration (invalid ones get key INT32_MAX and are counted).
__global__ void k_feedback_keys(DevProblem P, int64_t n, const int32_t *obs_op, const int32_t *obs_cfg,
                                const int32_t *obs_lat, const int64_t *obs_cost, int32_t *keys, int32_t *idx,
                                unsigned long long *rejected) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = obs_op[i], x = obs_cfg[i];
        bool ok = v >= 0 && v < P.n_ops;
        if (ok) ok = x >= 0 && x < P.cfg_off[v + 1] - P.cfg_off[v];
        ok = ok && obs_lat[i] >= 1 && obs_lat[i] < INT32_MAX && obs_cost[i] >= 0 && obs_cost[i] < (1ll << 46);
        keys[i] = ok ? (int32_t)(P.cfg_off[v] + x) : INT32_MAX;
        idx[i] = (int32_t)i;
        if (!ok) atomicAdd(rejected, 1ull);
    }
}

// Feedback, step 2: the first observation of every configuration (in key
// order, stable) applies all of that configuration's observations in their
// order: L <- ((b_den - b_num) L + b_num L_obs + b_den / 2) / b_den, the same
// for the cost, in exact integers.
__global__ void k_feedback_apply(DevProblem P, int64_t n, const int32_t *sorted_g, const int32_t *sorted_obs,
                                 const int32_t *obs_op, const int32_t *obs_lat, const int64_t *obs_cost,
                                 int32_t beta_num, int32_t beta_den, int32_t *lat, int64_t *cost,
                                 uint8_t *touched) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = sorted_g[k];
        if (g == INT32_MAX || (k > 0 && sorted_g[k - 1] == g)) continue;
        const int64_t w = beta_den - beta_num;
        int64_t L = lat[g], C = cost[g];
        int64_t j = k;
        for (; j < n && sorted_g[j] == g; ++j) {
            const int32_t o = sorted_obs[j];
            L = (w * L + (int64_t)beta_num * obs_lat[o] + beta_den / 2) / beta_den;
            C = (w * C + (int64_t)beta_num * obs_cost[o] + beta_den / 2) / beta_den;
        }
        lat[g] = (int32_t)min(max(L, (int64_t)1), (int64_t)INT32_MAX - 1);
        cost[g] = C;
        touched[obs_op[sorted_obs[k]]] = 1;
    }
}

// Feedback, step 4: the distinct-latency count of every re-encoded op in the
// bucket-order table.
__global__ void k_refresh_order(DevProblem P, const int32_t *ord_pos, int4 *ord_info) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= P.n_ops || !P.encode_only[v]) return;
    ord_info[ord_pos[v]].w = P.dlat_n[v];
}


// ---------------------------------------------------------------------------
// Serving loop: one tick of early speculation and late commit (Section 4.3)
// with priority-based commit (Section 4.4), by one CTA of 1024 threads; the
// state lives in device memory (LoopState, the slot arrays and the queues).
// ---------------------------------------------------------------------------

// Arrival-order ranks of one tick's admissions, in one pass (two barriers):
// for each thread, how many threads before it are valid (*vrank) and how many
// before it are valid and speculated onto its own backend lam (*hrank);
// tot[0] = valid ones, tot[1 + h] = those onto backend h.  cnt and pre hold
// (LLAMA_MAX_HW + 1) x 32 words; one warp per category scans the per-warp
// counts.  Every thread of the (1024-thread) block must call it.
__device__ __forceinline__ void block_admission_ranks(bool valid, int lam, int H, int *vrank, int *hrank,
                                                      int (*cnt)[32], int (*pre)[32], int *tot) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned below = (1u << lane) - 1u;
    const unsigned bv = __ballot_sync(0xffffffffu, valid);
    if (lane == 0) cnt[0][wid] = __popc(bv);
    unsigned mine = 0;
    for (int h = 0; h < H; ++h) {
        const unsigned b = __ballot_sync(0xffffffffu, valid && lam == h);
        if (lane == 0) cnt[1 + h][wid] = __popc(b);
        if (lam == h) mine = b;
    }
    __syncthreads();
    if (wid <= H) {  // warp k scans category k over the 32 warps
        const int c = cnt[wid][lane];
        int inc = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        pre[wid][lane] = inc - c;
        if (lane == 31) tot[wid] = inc;
    }
    __syncthreads();
    *vrank = pre[0][wid] + __popc(bv & below);
    *hrank = lam >= 0 ? pre[1 + lam][wid] + __popc(mine & below) : 0;
}

// Eq. 2 over both queues: floor(s / R_total), clamped at INT32_MAX (every sum
// at or above INT32_MAX * R_total clamps, and a smaller one fits 64 bits).
__device__ __forceinline__ int64_t loop_queue_time(unsigned __int128 s, int32_t r_total) {
    const unsigned __int128 cap = (unsigned __int128)INT32_MAX * (uint32_t)r_total;
    if (s >= cap) return INT32_MAX;
    return (int64_t)((uint64_t)s / (uint32_t)r_total);
}

__device__ __forceinline__ unsigned long long decision_lr(const DevProblem &P, int32_t g, const llama_decision &d) {
    return (unsigned long long)(uint32_t)d.lat * (unsigned long long)(uint32_t)P.res[P.cfg_off[g] + d.cfg];
}

__device__ __forceinline__ void loop_record(const LoopDev &L, long long *dropped, long long pos, long long res_read,
                                            int64_t id, int32_t kind, int32_t tick, const llama_decision &d,
                                            int32_t lam) {
    if (pos - res_read >= L.res_cap) {  // the host has not taken enough records: drop, count
        atomicAdd(reinterpret_cast<unsigned long long *>(dropped), 1ull);
        return;
    }
    llama_loop_result rec;
    rec.id = id;
    rec.kind = kind;
    rec.tick = tick;
    rec.decision = d;
    rec.backend = lam;
    rec.pad = 0;
    L.res[pos & (L.res_cap - 1)] = rec;
}

__global__ void __launch_bounds__(kLoopThreads) k_loop_tick(DevProblem P, LoopDev L, LoopTickArgs a) {
    const int H = P.n_hw, tid = threadIdx.x;
    // the loop's state is worked on in shared memory (the serial steps below
    // then touch no device memory) and written back at the end of the tick
    __shared__ __align__(16) LoopState S;
    constexpr int kStateWords = (int)(sizeof(LoopState) / 8);
    static_assert(sizeof(LoopState) % 8 == 0, "state copied in 8-byte words");
    for (int k = tid; k < kStateWords; k += kLoopThreads)
        reinterpret_cast<unsigned long long *>(&S)[k] = reinterpret_cast<const unsigned long long *>(L.st)[k];
    // the requests this tick may admit (at most max_admit of those submitted
    // before it), read from the mapped ring now so the host link's latency
    // overlaps the dispatch step; admission takes a prefix of them
    llama_loop_request r;
    r.id = 0;
    {
        const long long head = L.st->head;
        if (tid < L.max_admit && head + tid < a.limit) r = L.ring[(head + tid) & L.ring_mask];
    }
    __shared__ int adm_cnt[LLAMA_MAX_HW + 1][32], adm_pre[LLAMA_MAX_HW + 1][32], adm_tot[LLAMA_MAX_HW + 1];
    __shared__ int32_t sh_disp[LLAMA_MAX_HW];
    __shared__ int sh_n_adm, sh_free_top, sh_tick;
    __shared__ long long sh_res, sh_res_read;
    __shared__ long long sh_sq_head[LLAMA_MAX_HW], sh_sq_tail[LLAMA_MAX_HW], sh_cq_tail[LLAMA_MAX_HW];
    __shared__ int sh_room[LLAMA_MAX_HW], sh_cnt[LLAMA_MAX_HW], sh_w[LLAMA_MAX_HW + 1], sh_group[LLAMA_MAX_HW],
        sh_ncommit_src[LLAMA_MAX_HW];
    __shared__ unsigned long long sh_lr_in[LLAMA_MAX_HW], sh_lr_out[LLAMA_MAX_HW];
    // Eq. 3 affinities as order-preserving integer keys: non-negative doubles
    // (+inf included) compare as their bit patterns read as unsigned integers
    __shared__ unsigned long long c_aff[kLoopThreads];
    __shared__ int8_t c_lam[kLoopThreads], c_commit[kLoopThreads];
    // records the host has taken (mapped memory), read by the thread that uses it
    long long res_read = 0;
    if (tid == 0) res_read = (long long)*reinterpret_cast<volatile unsigned long long *>(&L.ctl->res_read);
#pragma unroll
    for (int h = 0; h < LLAMA_MAX_HW; ++h)  // constant indices into the argument
        if (tid == h) sh_disp[h] = a.dispatch[h];
    __syncthreads();  // the state copy is complete

    // 1. dispatch: the heads of the commit queues leave (their slots go back on
    //    the free stack in backend order, then queue order, so the stack's order
    //    is reproducible), a thread per dispatched invocation; then the
    //    queueing time at the tick's start (Eq. 2 over both queues)
    if (tid == 0) {
        int off = 0;
        for (int h = 0; h < H; ++h) {
            const long long len = S.cq_tail[h] - S.cq_head[h];
            const int k = (int)min((long long)max(sh_disp[h], 0), len);
            sh_cnt[h] = off;  // first dispatched entry of backend h
            off += k;
            sh_lr_out[h] = 0;
        }
        sh_w[0] = off;  // dispatched in all
        sh_free_top = S.free_top;
        for (int h = 0; h < H; ++h) sh_cq_tail[h] = S.cq_head[h];  // the heads, for the loop below
    }
    __syncthreads();
    {
        const int n_disp = sh_w[0];
        for (int t = tid; t < n_disp; t += kLoopThreads) {
            int h = 0;
            while (h + 1 < H && t >= sh_cnt[h + 1]) ++h;
            const long long pos = sh_cq_tail[h] + (t - sh_cnt[h]);
            const int32_t slot = L.cq[(int64_t)h * L.cq_stride + pos % L.cq_cap[h]];
            if (!LLAMA_IN_BOUNDS(P, slot >= 0 && slot < L.slots, LLAMA_CHECK_LOOP)) continue;
            atomicAdd(&sh_lr_out[h], L.slot_lr_commit[slot]);
            L.free_stack[sh_free_top + t] = slot;
        }
    }
    __syncthreads();
    if (tid == 0) {
        const int n_disp = sh_w[0];
        for (int h = 0; h < H; ++h) {
            const int k = (h + 1 < H ? sh_cnt[h + 1] : n_disp) - sh_cnt[h];
            S.s_cq[h] -= sh_lr_out[h];
            S.cq_head[h] += k;
        }
        S.dispatched += n_disp;
        const int32_t ft = S.free_top + n_disp;
        S.free_top = ft;
        for (int h = 0; h < H; ++h) L.q[h] = loop_queue_time(S.s_sq[h] + S.s_cq[h], P.res_total[h]);
        const long long avail = max(0ll, a.limit - S.head);
        sh_n_adm = (int)min(avail, (long long)min(ft, L.max_admit));
        sh_free_top = ft;
        sh_res = S.res_count;
        sh_tick = (int)S.ticks;
        sh_res_read = res_read;
        for (int h = 0; h < H; ++h) {
            sh_sq_head[h] = S.sq_head[h];
            sh_sq_tail[h] = S.sq_tail[h];
            sh_cq_tail[h] = S.cq_tail[h];
            sh_room[h] = L.cq_cap[h] - (int)(S.cq_tail[h] - S.cq_head[h]);
            sh_lr_in[h] = 0;
            sh_lr_out[h] = 0;
            sh_group[h] = 0;
            sh_ncommit_src[h] = 0;
            sh_cnt[h] = 0;
        }
    }
    __syncthreads();

    // 2. admit in arrival order and speculate (Algorithm 1 under the queueing
    //    time at the tick's start, Eq. 1 through the staircase tables)
    const int n_adm = sh_n_adm;
    bool valid = false;
    int lam = -1;
    llama_decision dsn;
    dsn.cfg = -1;
    dsn.lat = 0;
    dsn.cost = 0;
    dsn.slack = 0;
    dsn.flags = LLAMA_FLAG_INVALID;
    unsigned long long lr = 0;
    if (tid < n_adm) {
        int32_t g;
        int64_t rbase;
        if (invocation_op(P, r.dag, r.op_local, r.start_us, a.now, g, rbase)) {
            valid = true;
            dsn = stair_decide(P, g, rbase, &lam);
            lr = decision_lr(P, g, dsn);
        }
    }
    // ranks among this tick's valid admissions, and among those speculated onto
    // the same backend
    int vrank, hrank;
    block_admission_ranks(valid, valid ? lam : -1, H, &vrank, &hrank, adm_cnt, adm_pre, adm_tot);
    const int n_valid = adm_tot[0];
    if (tid < H) sh_cnt[tid] = adm_tot[1 + tid];
    if (valid) {
        const int32_t slot = L.free_stack[sh_free_top - 1 - vrank];
        L.slot_id[slot] = r.id;
        L.slot_dag[slot] = r.dag;
        L.slot_opl[slot] = r.op_local;
        L.slot_start[slot] = r.start_us;
        L.slot_lr_spec[slot] = lr;
        L.sq[(int64_t)lam * L.slots + (sh_sq_tail[lam] + hrank) % L.slots] = slot;
        atomicAdd(&sh_lr_in[lam], lr);
    }
    if (tid < n_adm)
        loop_record(L, &S.dropped, sh_res + tid, sh_res_read, r.id, valid ? LLAMA_LOOP_SPECULATED : LLAMA_LOOP_REJECTED,
                    sh_tick, dsn, lam);
    __syncthreads();
    if (tid == 0) {
        for (int h = 0; h < H; ++h) {
            S.s_sq[h] += sh_lr_in[h];
            S.sq_tail[h] += sh_cnt[h];
            sh_sq_tail[h] += sh_cnt[h];
            sh_lr_in[h] = 0;
        }
        S.free_top = sh_free_top - n_valid;
        S.head += n_adm;
        S.res_count += n_adm;
        S.admitted += n_valid;
        S.rejected += n_adm - n_valid;
        sh_res = S.res_count;
        // the queueing time after speculation: what the revisited heads see
        for (int h = 0; h < H; ++h) L.q[h] = loop_queue_time(S.s_sq[h] + S.s_cq[h], P.res_total[h]);
        int c = 0;
        for (int h = 0; h < H; ++h) {
            sh_w[h] = c;
            c += (int)min(sh_sq_tail[h] - sh_sq_head[h], (long long)L.cq_cap[h]);
        }
        sh_w[H] = c;
    }
    __syncthreads();

    // 3. late commit: the heads of every speculative queue, re-scored together
    //    (Algorithm 1 and Eq. 1 again, at the tick's time)
    const int C = sh_w[H];
    int src = 0, lam2 = -1;
    int32_t slot = -1, g2 = 0;
    llama_decision d2 = dsn;
    if (tid < C) {
        while (src + 1 < H && tid >= sh_w[src + 1]) ++src;
        slot = L.sq[(int64_t)src * L.slots + (sh_sq_head[src] + (tid - sh_w[src])) % L.slots];
        if (!LLAMA_IN_BOUNDS(P, slot >= 0 && slot < L.slots, LLAMA_CHECK_LOOP)) slot = 0;
        const int32_t d = L.slot_dag[slot];
        g2 = P.dag_op_off[d] + L.slot_opl[slot];
        const long long rb = P.slo[d] - (a.now - L.slot_start[slot]);
        int32_t cnt[LLAMA_MAX_HW];
        d2 = stair_decide(P, g2, rb, &lam2, cnt);
        // Eq. 3: the least objective per backend under the same slacks, from
        // the minima tables at the counts the decision searched
        const int64_t *om = L.objmin + P.stair_off[g2];
        const int64_t stride = P.cfg_off[g2 + 1] - P.cfg_off[g2] + 1;
        int64_t best[LLAMA_MAX_HW];
#pragma unroll
        for (int h = 0; h < LLAMA_MAX_HW; ++h) best[h] = h < H ? __ldg(om + h * stride + cnt[h]) : INT64_MAX;
        c_aff[tid] = (unsigned long long)__double_as_longlong(affinity_of(best, H, lam2));
        c_lam[tid] = (int8_t)lam2;
    }
    __syncthreads();
    // the commit order: by backend, descending affinity, then candidate order
    int rank = 0;
    if (tid < C) {
        const unsigned long long my = c_aff[tid];
        for (int k = 0; k < C; ++k) {
            if (c_lam[k] != lam2) continue;
            const unsigned long long o = c_aff[k];
            rank += (o > my) || (o == my && k < tid);
        }
        atomicAdd(&sh_group[lam2], 1);
    }
    const bool commit = tid < C && rank < sh_room[lam2 < 0 ? 0 : lam2];
    if (tid < C) c_commit[tid] = commit ? 1 : 0;
    __syncthreads();
    if (commit) {
        int before = 0;  // commits of the backends before lam2 (their records come first)
        for (int t = 0; t < lam2; ++t) before += min(sh_group[t], max(sh_room[t], 0));
        L.cq[(int64_t)lam2 * L.cq_stride + (sh_cq_tail[lam2] + rank) % L.cq_cap[lam2]] = slot;
        const unsigned long long lr2 = decision_lr(P, g2, d2);
        L.slot_lr_commit[slot] = lr2;
        atomicAdd(&sh_lr_in[lam2], lr2);
        atomicAdd(&sh_lr_out[src], L.slot_lr_spec[slot]);
        atomicAdd(&sh_ncommit_src[src], 1);
        loop_record(L, &S.dropped, sh_res + before + rank, sh_res_read, L.slot_id[slot], LLAMA_LOOP_COMMITTED, sh_tick,
                    d2, lam2);
    }
    __syncthreads();
    if (tid < C && !commit) {
        // a candidate that stays keeps its place behind the ones removed before it
        int u = 0;
        for (int k = sh_w[src]; k < tid; ++k) u += c_commit[k] ? 0 : 1;
        L.sq[(int64_t)src * L.slots + (sh_sq_head[src] + sh_ncommit_src[src] + u) % L.slots] = slot;
    }
    __threadfence_system();  // records before the count that publishes them
    __syncthreads();
    if (tid == 0) {
        long long n_commit = 0;
        for (int h = 0; h < H; ++h) {
            const int k = min(sh_group[h], max(sh_room[h], 0));
            S.s_cq[h] += sh_lr_in[h];
            S.s_sq[h] -= sh_lr_out[h];
            S.sq_head[h] += sh_ncommit_src[h];
            S.cq_tail[h] += k;
            n_commit += k;
        }
        S.committed += n_commit;
        S.res_count += n_commit;
        S.ticks += 1;
        volatile LoopCtl *ctl = L.ctl;
        ctl->head = (unsigned long long)S.head;
        ctl->dropped = (unsigned long long)S.dropped;
        ctl->inflight = (unsigned long long)(S.admitted - S.dispatched);
        ctl->ticks = (unsigned long long)S.ticks;
        __threadfence_system();
        ctl->res_count = (unsigned long long)S.res_count;
    }
    __syncthreads();
    for (int k = tid; k < kStateWords; k += kLoopThreads)
        reinterpret_cast<unsigned long long *>(L.st)[k] = reinterpret_cast<const unsigned long long *>(&S)[k];
}

cudaError_t enqueue_loop_tick(const DevProblem &P, const LoopDev &L, const LoopTickArgs &a, cudaStream_t s) {
    k_loop_tick<<<1, kLoopThreads, 0, s>>>(P, L, a);
    return cudaGetLastError();
}

cudaError_t enqueue_critical_paths(const ContextView &v, cudaStream_t s) {
    k_critical_paths<<<std::max(1, (v.n_dags + 7) / 8), 256, 0, s>>>(v.P, v.topo, v.lvl_off, v.dag_lvl);
    return cudaGetLastError();
}

}  // namespace llama
