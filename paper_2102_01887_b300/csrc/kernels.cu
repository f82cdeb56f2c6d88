// kernels.cu -- sm_103a kernels of the scheduling step.
//
//   k_critical_path   longest remaining reference-latency path per op (Alg. 1's
//                     RemainingPathLatency maximised over paths), one CTA per DAG,
//                     level-synchronous from the sinks upwards.
//   k_bucket_count    validate invocations, count them per operation.
//   k_bucket_scan     exclusive prefix of the counts and of the scan work.
//   k_bucket_scatter  bucket invocations by operation and compute their slack per
//                     backend (Algorithm 1 through the critical path).
//   k_score           Eq. 1 over every configuration of each invocation's operation
//                     and the argmin, on the rank-encoded tables staged in shared memory.
//   k_encode_*        build the rank encoding of the tables (once per llama_set_profiles).
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
// a1: critical path
// ---------------------------------------------------------------------------

__global__ void k_critical_path(DevProblem P, const int32_t *topo, const int32_t *lvl_off,
                                const int32_t *dag_lvl) {
    const int d = blockIdx.x;
    const int lo = P.dag_op_off[d], hi = P.dag_op_off[d + 1];
    for (int v = lo + (int)threadIdx.x; v < hi; v += blockDim.x)
        P.ref[v] = (int64_t)P.lat[P.cfg_off[v] + P.ref_cfg[v]];
    __syncthreads();
    // Levels hold the ops of equal height above the sinks (height 0 first), so
    // every successor's value is final before its predecessors read it.
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

// ---------------------------------------------------------------------------
// a3: bucketing (with a2 fused into the scatter)
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool invocation_valid(const DevProblem &P, int32_t d, int32_t o,
                                                 int64_t s, int64_t now) {
    if (d < 0 || d >= P.n_dags) return false;
    if (o < 0 || o >= P.dag_op_off[d + 1] - P.dag_op_off[d]) return false;
    return s >= 0 && s <= now;
}

__global__ void k_bucket_count(DevProblem P, int64_t n_inv, const int32_t *dag,
                               const int32_t *op_local, const int64_t *start, int64_t now,
                               BucketScratch S, llama_decision *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_inv;
         i += (int64_t)gridDim.x * blockDim.x) {
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
            atomicAdd(S.n_invalid, 1ull);
            continue;
        }
        const int32_t g = P.dag_op_off[d] + o;
        S.gop[i] = g;
        S.slot[i] = atomicAdd(&S.cnt[g], 1);
    }
}

// Single CTA: exclusive prefix of cnt and of cnt * padded table size.
__global__ void k_bucket_scan(DevProblem P, BucketScratch S) {
    __shared__ int32_t warp_c[32];
    __shared__ int64_t warp_w[32];
    const int n = P.n_ops, T = blockDim.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int per = (n + T - 1) / T;
    const int b = min(n, tid * per), e = min(n, b + per);
    int32_t c = 0;
    int64_t w = 0;
    for (int k = b; k < e; ++k) {
        const int32_t ck = S.cnt[k];
        c += ck;
        w += (int64_t)ck * (P.pad_off[k + 1] - P.pad_off[k]);
    }
    // inclusive warp scan
    int32_t ci = c;
    int64_t wi = w;
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t cu = __shfl_up_sync(0xffffffffu, ci, o);
        const int64_t wu = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) { ci += cu; wi += wu; }
    }
    if (lane == 31) { warp_c[wid] = ci; warp_w[wid] = wi; }
    __syncthreads();
    if (wid == 0) {
        const int nw = T >> 5;
        int32_t cw = lane < nw ? warp_c[lane] : 0;
        int64_t ww = lane < nw ? warp_w[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t cu = __shfl_up_sync(0xffffffffu, cw, o);
            const int64_t wu = __shfl_up_sync(0xffffffffu, ww, o);
            if (lane >= o) { cw += cu; ww += wu; }
        }
        if (lane < nw) { warp_c[lane] = cw; warp_w[lane] = ww; }
    }
    __syncthreads();
    int32_t c0 = ci - c + (wid > 0 ? warp_c[wid - 1] : 0);
    int64_t w0 = wi - w + (wid > 0 ? warp_w[wid - 1] : 0);
    for (int k = b; k < e; ++k) {
        S.op_start[k] = c0;
        S.wprefix[k] = w0;
        const int32_t ck = S.cnt[k];
        c0 += ck;
        w0 += (int64_t)ck * (P.pad_off[k + 1] - P.pad_off[k]);
    }
    if (tid == T - 1) {
        S.op_start[n] = c0;
        S.wprefix[n] = w0;
    }
}

__global__ void k_bucket_scatter(DevProblem P, int64_t n_inv, const int32_t *dag,
                                 const int64_t *start, int64_t now, BucketScratch S) {
    const int H = P.n_hw;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_inv;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = S.gop[i];
        if (g < 0) continue;
        const int32_t pos = S.op_start[g] + S.slot[i];
        S.b_inv[pos] = (int32_t)i;
        const int64_t r_base = P.slo[dag[i]] - (now - start[i]);
        const int64_t ref = P.ref[g], cp = P.cp[g];
        for (int h = 0; h < H; ++h)
            S.b_slack[(int64_t)pos * H + h] = slack_of(ref, cp, r_base - P.q[h]);
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

// Lanes per invocation (1..32, a power of two) for m invocations of an op on T
// threads: minimise rounds x (vector iterations per lane + per-invocation
// overhead + shuffle levels).  Uniform over the CTA.
__device__ __forceinline__ int pick_lanes(int m, int T, const int32_t *seg_s, int H) {
    int best_l = 1;
    long long best_cost = LLONG_MAX;
    int lg = 0;
    for (int l = 1; l <= 32; l <<= 1, ++lg) {
        const int groups = T / l;
        const int rounds = (m + groups - 1) / groups;
        int iters = 0;
        for (int h = 0; h < H; ++h) {
            const int nv = (seg_s[h + 1] - seg_s[h]) / kVec;
            iters += (nv + l - 1) / l;
        }
        const long long cost = (long long)rounds * (iters + 6 + 2 * lg);
        if (cost < best_cost) { best_cost = cost; best_l = l; }
    }
    return best_l;
}

// Persistent CTAs split the total scan work (sum over ops of invocations x
// padded table size) into equal contiguous ranges; a CTA walks the ops its
// range covers, stages each op's encoded table into shared memory once and
// scores all of that op's invocations in its range against it.
template <int MODE>
__device__ __forceinline__ void score_body(const DevProblem &P, const BucketScratch &S,
                                           llama_decision *out, unsigned char *smem_raw,
                                           int32_t *seg_s) {
    const int T = blockDim.x, tid = threadIdx.x;
    const int H = P.n_hw;
    const int64_t W = S.wprefix[P.n_ops];
    const int64_t w_lo = W * blockIdx.x / gridDim.x;
    const int64_t w_hi = W * (blockIdx.x + 1) / gridDim.x;
    if (w_lo >= w_hi) return;

    int32_t *lat_s = reinterpret_cast<int32_t *>(smem_raw);
    const int cap = P.max_npad;
    uint16_t *rf_s = reinterpret_cast<uint16_t *>(smem_raw + 4 * (size_t)cap);
    uint16_t *df_s = rf_s + cap;

    int lo = 0, hi = P.n_ops - 1;  // largest v with wprefix[v] <= w_lo
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (S.wprefix[mid] <= w_lo) lo = mid; else hi = mid - 1;
    }
    for (int v = lo; v < P.n_ops; ++v) {
        const int64_t wp = S.wprefix[v];
        if (wp >= w_hi) break;
        const int32_t c0 = S.op_start[v];
        const int32_t cnt = S.op_start[v + 1] - c0;
        if (cnt == 0) continue;
        const int64_t p0 = P.pad_off[v];
        const int32_t npad = (int32_t)(P.pad_off[v + 1] - p0);
        const int64_t rlo = w_lo - wp, rhi = w_hi - wp;
        const int32_t j0 = rlo <= 0 ? 0 : (int32_t)((rlo + npad - 1) / npad);
        const int64_t j1_raw = (rhi + npad - 1) / npad;
        const int32_t j1 = j1_raw < cnt ? (int32_t)j1_raw : cnt;
        if (j0 >= j1) continue;

        __syncthreads();  // the previous op's table is no longer read
        {
            const uint4 *src = reinterpret_cast<const uint4 *>(P.lat_pad + p0);
            uint4 *dst = reinterpret_cast<uint4 *>(lat_s);
            for (int k = tid; k < npad / 4; k += T) dst[k] = src[k];
            const uint4 *srf = reinterpret_cast<const uint4 *>(P.rf + p0);
            uint4 *drf = reinterpret_cast<uint4 *>(rf_s);
            for (int k = tid; k < npad / 8; k += T) drf[k] = srf[k];
            if (MODE == LLAMA_MODE_ALPHA) {
                const uint4 *sdf = reinterpret_cast<const uint4 *>(P.df + p0);
                uint4 *ddf = reinterpret_cast<uint4 *>(df_s);
                for (int k = tid; k < npad / 8; k += T) ddf[k] = sdf[k];
            }
            if (tid <= H) seg_s[tid] = P.seg_pad[(int64_t)v * (H + 1) + tid];
        }
        __syncthreads();

        const int m = j1 - j0;
        const int lanes = pick_lanes(m, T, seg_s, H);
        const int groups = T / lanes;
        const int g = tid / lanes, s = tid % lanes;
        const int rounds = (m + groups - 1) / groups;
        const int4 *lat4 = reinterpret_cast<const int4 *>(lat_s);
        const uint4 *rf4 = reinterpret_cast<const uint4 *>(rf_s);
        const uint4 *df4 = reinterpret_cast<const uint4 *>(df_s);

        for (int r = 0; r < rounds; ++r) {
            const int j = j0 + r * groups + g;
            const bool active = j < j1;
            const int32_t pos = c0 + j;
            uint32_t key = 0xFFFFu;
            if (active) {
                uint32_t best = 0xFFFFFFFFu;
                for (int h = 0; h < H; ++h) {
                    // t = (slack - 1) - L is negative exactly when L >= slack (infeasible)
                    const int32_t sm1 = S.b_slack[(int64_t)pos * H + h] - 1;
                    const int qa = seg_s[h] / kVec, qb = seg_s[h + 1] / kVec;
                    for (int q = qa + s; q < qb; q += lanes) {
                        const int4 l0 = lat4[2 * q], l1 = lat4[2 * q + 1];
                        const uint4 rk = rf4[q];
                        const uint32_t t0 = (uint32_t)(sm1 - l0.x), t1 = (uint32_t)(sm1 - l0.y);
                        const uint32_t t2 = (uint32_t)(sm1 - l0.z), t3 = (uint32_t)(sm1 - l0.w);
                        const uint32_t t4 = (uint32_t)(sm1 - l1.x), t5 = (uint32_t)(sm1 - l1.y);
                        const uint32_t t6 = (uint32_t)(sm1 - l1.z), t7 = (uint32_t)(sm1 - l1.w);
                        if (MODE == LLAMA_MODE_ALPHA) {
                            // sign bytes replicated: 0xFFFF in a half where that config is infeasible
                            const uint4 dk = df4[q];
                            best = vmin_u16x2(best, rk.x ^ (dk.x & prmt(t0, t1, 0xFFBBu)));
                            best = vmin_u16x2(best, rk.y ^ (dk.y & prmt(t2, t3, 0xFFBBu)));
                            best = vmin_u16x2(best, rk.z ^ (dk.z & prmt(t4, t5, 0xFFBBu)));
                            best = vmin_u16x2(best, rk.w ^ (dk.w & prmt(t6, t7, 0xFFBBu)));
                        } else {
                            // sign bits moved to bits 15 and 31: infeasible keys get 0x8000 added
                            best = vmin_u16x2(best, rk.x | (prmt(t0, t1, 0x7430u) & 0x80008000u));
                            best = vmin_u16x2(best, rk.y | (prmt(t2, t3, 0x7430u) & 0x80008000u));
                            best = vmin_u16x2(best, rk.z | (prmt(t4, t5, 0x7430u) & 0x80008000u));
                            best = vmin_u16x2(best, rk.w | (prmt(t6, t7, 0x7430u) & 0x80008000u));
                        }
                    }
                }
                key = min(best & 0xFFFFu, best >> 16);
            }
            for (int o = 1; o < lanes; o <<= 1) key = min(key, __shfl_xor_sync(0xffffffffu, key, o));
            if (active && s == 0) {
                const int32_t i = S.b_inv[pos];
                const int64_t c_base = P.cfg_off[v];
                int32_t idx;
                if (MODE == LLAMA_MODE_ALPHA) idx = P.inv[2 * c_base + key];
                else idx = key < 0x8000u ? (int32_t)P.inv[2 * c_base + key] : P.fast[v];
                const int64_t gx = c_base + idx;
                const int32_t L = P.lat[gx];
                const int lam = backend_of(P.hw_off + (int64_t)v * (H + 1), H, idx);
                const int32_t sl = S.b_slack[(int64_t)pos * H + lam];
                llama_decision dsn;
                dsn.cfg = idx;
                dsn.lat = L;
                dsn.cost = P.cost[gx];
                dsn.slack = sl;
                dsn.flags = L < sl ? LLAMA_FLAG_FEASIBLE : 0;
                out[i] = dsn;
            }
        }
    }
}

__global__ void __launch_bounds__(kScoreThreads)
    k_score_cost_first(DevProblem P, BucketScratch S, llama_decision *out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int32_t seg_s[LLAMA_MAX_HW + 1];
    score_body<LLAMA_MODE_COST_FIRST>(P, S, out, smem_raw, seg_s);
}

__global__ void __launch_bounds__(kScoreThreads)
    k_score_alpha(DevProblem P, BucketScratch S, llama_decision *out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int32_t seg_s[LLAMA_MAX_HW + 1];
    score_body<LLAMA_MODE_ALPHA>(P, S, out, smem_raw, seg_s);
}

// ---------------------------------------------------------------------------
// Encoding of the tables (llama_set_profiles)
// ---------------------------------------------------------------------------

// One CTA per op: latencies into the padded layout (INT32_MAX at pads, which no
// slack can exceed), ranks initialised to the pad rank, and the op's fastest
// configuration argmin (L, index).
__global__ void k_encode_pad(DevProblem P, int32_t *lat_pad, uint16_t *rf, uint16_t *df,
                             int32_t *fast) {
    __shared__ int64_t red[32];
    const int v = blockIdx.x, H = P.n_hw;
    const int64_t c0 = P.cfg_off[v], p0 = P.pad_off[v];
    const int32_t *hw = P.hw_off + (int64_t)v * (H + 1);
    const int32_t *sp = P.seg_pad + (int64_t)v * (H + 1);
    for (int h = 0; h < H; ++h) {
        const int src_n = hw[h + 1] - hw[h], dst_n = sp[h + 1] - sp[h];
        for (int k = threadIdx.x; k < dst_n; k += blockDim.x) {
            const int64_t dst = p0 + sp[h] + k;
            lat_pad[dst] = k < src_n ? P.lat[c0 + hw[h] + k] : INT32_MAX;
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
