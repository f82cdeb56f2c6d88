// Dense BF16 GEMM on the 5th-generation tensor cores (tcgen05), FP32
// accumulation in tensor memory: C[M x N] = A[M x K] . B[N x K]^T (+ bias[N],
// optionally ReLU), both operands K-major.  The building block of the learned
// latency surrogate (a 4-layer MLP of width 256).
//
// One CTA computes a 128 x BN tile.  Warp 0 (one lane) streams 128 x 64 and
// BN x 64 operand tiles into a ring of shared-memory stages with TMA (128-byte
// swizzle); warp 1 (one lane) issues tcgen05.mma (M 128, N BN, K 16, four per
// stage) into a 128 x BN FP32 accumulator in tensor memory and releases each
// stage with tcgen05.commit; the four warps then read the accumulator back
// (tcgen05.ld, warp w owns rows 32w..32w+31), add the bias, apply ReLU and store
// BF16 and/or FP32.  Every wait is bounded: a wait that gives up sets *err and
// the CTA still waits (bounded) for its copies and MMAs in flight and frees its
// tensor memory before it returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "llama_surrogate.h"
#include "sg_internal.cuh"

namespace sgk {

constexpr int kBM = 128;            // rows per tile (tensor-memory lanes)
constexpr int kBK = 64;             // K per stage: one 128-byte swizzle row of BF16
constexpr int kStages = 4;
constexpr int kThreads = 128;
constexpr int kMaxTries = 1 << 22;  // bounded mbarrier waits
static_assert(kBM == kTileRows, "the pair layers' tiles are the GEMM's row tiles");

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (int it = 0; it < kMaxTries; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar) : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart (descriptor version 1).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFF) >> 4)      // start address
           | ((uint64_t)1 << 16)                  // leading byte offset (unused here)
           | ((uint64_t)(1024 >> 4) << 32)        // stride byte offset
           | ((uint64_t)1 << 46)                  // version
           | ((uint64_t)2 << 61);                 // 128-byte swizzle
}

// Instruction descriptor of kind::f16: BF16 x BF16 -> FP32, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// Epilogue of the last hidden layer of the surrogate over (invocation,
// configuration) pairs (k_mlp_layer<true>): per row, h3 = ReLU(acc + bias), the log latency factor
// r = h3 . w4 + b4, the predicted latency and cost (profiled values times e^r)
// and the pair's selection key, folded into the invocation's best key.  The
// prediction is raised by the margin (an upper quantile of the model's error)
// before use.
// ps is the pair's selection record (invocation, op-local index, profiled
// latency, slack on its backend), cost its profiled cost.
__device__ __forceinline__ void select_row(const SelectArgs &A, int64_t row, float r, int4 ps, int64_t cost) {
    if (!isfinite(r)) r = 0.f;  // the profiled latency stands in for an unusable prediction
    r = fminf(fmaxf(r + A.margin, -20.f), 20.f);
    const int32_t i = ps.x, x = ps.y, sl = ps.w;
    const double f = (double)expf(r);
    const double lh = fmin(fmax(rint((double)ps.z * f), 1.0), 2147483646.0);
    const int32_t lhat = (int32_t)lh;
    const int64_t chat = (int64_t)fmin(rint((double)cost * f), 4.0e12);
    A.lhat[row] = lhat;
    A.chat[row] = chat;
    // cost-first: feasible pairs by (cost, index), else (latency, index) above them
    const unsigned long long key = lhat < sl ? ((unsigned long long)chat << 13) | (unsigned long long)x
                                             : (1ull << 62) | ((unsigned long long)lhat << 13) | (unsigned long long)x;
    atomicMin(A.best + i, key);
}

template <int BN>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_bf16(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N,
                int K, const float *__restrict__ bias, int flags, __nv_bfloat16 *__restrict__ c16,
                float *__restrict__ c32, int ldc, int *err) {
    constexpr int A_BYTES = kBM * kBK * 2, B_BYTES = BN * kBK * 2, STAGE = A_BYTES + B_BYTES;
    constexpr uint32_t TMEM_COLS = BN < 32 ? 32 : BN;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], accf;
    __shared__ uint32_t tmem_slot;
    __shared__ int issued, consumed, failed;
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // split K (gridDim.z > 1): CTA z takes K blocks [z * nk, (z + 1) * nk) and
    // writes its FP32 partial product to slice z of c32 (M x ldc each)
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN, nk = K / kBK / (int)gridDim.z;
    const int kb0 = (int)blockIdx.z * nk;
    if (c32) c32 += (int64_t)blockIdx.z * M * ldc;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        mbar_init(smem_u32(&accf), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        issued = consumed = failed = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_slot)), "r"(TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer: TMA into the stage ring
        int kb = 0;
        for (; kb < nk; ++kb) {
            const int s = kb % kStages;
            if (kb >= kStages && !mbar_wait(smem_u32(&empty[s]), ((kb / kStages) - 1) & 1)) {
                failed = 1;
                break;
            }
            const uint32_t a = base + s * STAGE, b = a + A_BYTES, bar = smem_u32(&full[s]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(STAGE) : "memory");
            tma_load_2d(a, &tmA, (kb0 + kb) * kBK, m0, bar);
            tma_load_2d(b, &tmB, (kb0 + kb) * kBK, n0, bar);
        }
        issued = kb;
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_bf16(kBM, BN);
        int kb = 0;
        for (; kb < nk; ++kb) {
            const int s = kb % kStages;
            if (!mbar_wait(smem_u32(&full[s]), (kb / kStages) & 1)) {
                failed = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a = base + s * STAGE, b = a + A_BYTES;
#pragma unroll
            for (int j = 0; j < kBK / 16; ++j) {
                const uint64_t ad = smem_desc_sw128(a + 32 * j), bd = smem_desc_sw128(b + 32 * j);
                const uint32_t acc = (kb > 0 || j > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                    ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"(smem_u32(&empty[s])) : "memory");
        }
        consumed = kb;
        // completes once every MMA issued above has completed
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(smem_u32(&accf)) : "memory");
    }
    __syncwarp();
    // epilogue: thread (warp w, lane l) owns row m0 + 32w + l, tensor-memory lane 32w + l
    const bool acc_ok = mbar_wait(smem_u32(&accf), 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    const bool ok = acc_ok && !failed && nk > 0;
    const int row = m0 + warp * 32 + lane;
    const bool relu = flags & LLAMA_GEMM_RELU;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t r[16];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (!ok || row >= M) continue;
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            v[j] = __uint_as_float(r[j]) + (bias ? bias[n0 + c0 + j] : 0.f);
            if (relu) v[j] = fmaxf(v[j], 0.f);
        }
        const int64_t o = (int64_t)row * ldc + n0 + c0;
        if (c32) {
#pragma unroll
            for (int j = 0; j < 16; j += 4)
                *reinterpret_cast<float4 *>(c32 + o + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        }
        if (c16) {
            uint32_t p[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                p[j] = *reinterpret_cast<const uint32_t *>(&h);
            }
            *reinterpret_cast<uint4 *>(c16 + o) = make_uint4(p[0], p[1], p[2], p[3]);
            *reinterpret_cast<uint4 *>(c16 + o + 8) = make_uint4(p[4], p[5], p[6], p[7]);
        }
    }
    if (!ok) {
        if (threadIdx.x == 0) {
            atomicOr(err, 1);
            // copies issued but never consumed: let them land before the CTA exits
            for (int kb = consumed; kb < issued; ++kb)
                mbar_wait(smem_u32(&full[kb % kStages]), (kb / kStages) & 1);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// ---------------------------------------------------------------------------
// Persistent hidden layer of the surrogate: C[M x 256] = ReLU(A[M x 256] . W^T + b)
// ---------------------------------------------------------------------------
//
// For the pair layers of the scheduling path (M in the millions, N = K = 256):
// one CTA per SM loads W (256 x 256 BF16, 128 KB, four 256 x 64 slices with the
// 128-byte swizzle) into shared memory once and keeps it; warp 0 (one lane)
// streams the A tiles of the CTA's row tiles (blockIdx.x, + gridDim.x, ...)
// through a ring of 128 x 64 slices; warp 1 (one lane) issues the MMAs of a tile
// into one of two 128 x 256 FP32 accumulators in tensor memory (512 columns)
// and commits; the epilogue warps read an accumulator back (warp w: tensor-memory
// lanes 32(w%4) .. 32(w%4)+31), add the bias, apply ReLU and store BF16 rows
// or, for the last hidden layer, fold every row into the last layer's dot
// product and the selection (eight warps, two per lane quarter, each half of the
// columns; the halves of a row's dot product meet in shared memory); then they
// release the accumulator, so the next tile's MMAs overlap this tile's
// epilogue.  Every wait is bounded; a wait that gives up sets *err, and the CTA
// waits (bounded) for its copies and MMAs in flight and frees its tensor memory
// before it returns.
//
// Layer 2 (kLayerFirst) builds its A operand itself: the first layer splits by
// linearity into a configuration part (BF16 rows of n_cfg x 256) and an
// invocation part (FP32 rows of n_inv x 256, bias included), and the pair rows
// are laid out so that every 128-row tile holds consecutive configurations of
// one invocation's operation.  Warp 0 loads the tile's configuration rows with
// TMA into the operand ring; eight converter warps add the invocation's row,
// apply ReLU and write the BF16 result back in place (same swizzled layout);
// only then does warp 1 issue the MMAs on that slice.
//
// Warp 0 TMA, warp 1 MMA, then the epilogue warps, then the converter warps.
constexpr int kLayerSelect = 1;  // A rows from a BF16 matrix; last layer and selection
constexpr int kLayerFirst = 2;   // A rows built from the split first layer; BF16 rows out
__host__ __device__ constexpr int epi_warps() { return 8; }
__host__ __device__ constexpr int conv_warps(int mode) { return mode == kLayerFirst ? 8 : 0; }
constexpr int kConvPasses = kBM / 8 / 4;  // four rows per pass, kBM / 8 rows per converter warp
constexpr int kEpiBarrier = 1;   // named barrier of the epilogue warps (0 is __syncthreads)
constexpr int kConvBarrier = 2;  // named barrier of the converter warps
__host__ __device__ constexpr int layer_threads(int mode) { return 32 * (2 + epi_warps() + conv_warps(mode)); }
constexpr int kLStagesMax = 5;            // A ring of 128 x 64 BF16 slices
constexpr int kLSlices = kHid / kBK;      // K slices per tile (4)
constexpr int kLWSlice = kHid * kBK * 2;  // 256 x 64 BF16 = 32 KB
constexpr int kLWBytes = kLSlices * kLWSlice;
constexpr int kLABytes = kBM * kBK * 2;   // 16 KB
// kLayerFirst stages its output through shared memory (a 32 x 32 BF16 block
// per epilogue warp, stored by TMA) and keeps one A slice fewer for it
constexpr int kLStageBytes = 32 * 32 * 2;
__host__ __device__ constexpr int layer_stages(int mode) { return mode == kLayerFirst ? 4 : kLStagesMax; }
__host__ __device__ constexpr int layer_smem(int mode) {
    return kLWBytes + layer_stages(mode) * kLABytes + (mode == kLayerFirst ? epi_warps() * kLStageBytes : 0) + 1024;
}

// All lanes of the warp agree: true only if every lane's bounded wait completed.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity) {
    return __all_sync(0xffffffffu, mbar_wait(bar, parity));
}

// One 16-byte unit (eight BF16 columns) of a swizzled slice: ReLU(a + b) with
// b the invocation part of those columns, in BF16 pairs: a * 1 + b rounded once
// to BF16, negative results clamped to 0 (one instruction per two columns).
__device__ __forceinline__ uint4 relu_add_unit(uint4 a, uint4 b) {
    constexpr uint32_t one = 0x3F803F80u;  // (1, 1) in BF16
    uint4 r;
    asm("fma.rn.relu.bf16x2 %0, %1, %2, %3;" : "=r"(r.x) : "r"(a.x), "r"(one), "r"(b.x));
    asm("fma.rn.relu.bf16x2 %0, %1, %2, %3;" : "=r"(r.y) : "r"(a.y), "r"(one), "r"(b.y));
    asm("fma.rn.relu.bf16x2 %0, %1, %2, %3;" : "=r"(r.z) : "r"(a.z), "r"(one), "r"(b.z));
    asm("fma.rn.relu.bf16x2 %0, %1, %2, %3;" : "=r"(r.w) : "r"(a.w), "r"(one), "r"(b.w));
    return r;
}

template <int MODE>
__global__ void __launch_bounds__(layer_threads(MODE), 1)
    k_mlp_layer(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmW,
                const __grid_constant__ CUtensorMap tmC, int M, const float *__restrict__ bias,
                __nv_bfloat16 *__restrict__ c16, int *err,
                const __grid_constant__ SelectArgs sel, const int2 *__restrict__ tile_info,
                const float4 *__restrict__ b_inv) {
    constexpr bool SELECT = MODE == kLayerSelect, FIRST = MODE == kLayerFirst;
    constexpr int kLStages = layer_stages(MODE);
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[kLStages], empty[kLStages], ready[FIRST ? kLStages : 1], wbar, accf[2],
        acce[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int failed, issued, consumed, committed;
    __shared__ float half_dot[SELECT ? kBM : 1];  // second halves of the rows' last-layer dot products
    __shared__ __align__(16) float s_bias[kHid];
    __shared__ __align__(16) float s_w4[SELECT ? kHid : 4];
    // invocation part of this and the last tile in BF16, columns in order (the
    // eight columns of unit u of K-slice k, 64k + 8u .. 64k + 8u + 7, are the
    // 16-byte word 8k + u)
    __shared__ __align__(16) uint2 s_binv[FIRST ? 2 : 1][kHid / 4];
    const uint32_t wbase = (smem_u32(smem_raw) + 1023u) & ~1023u, abase = wbase + kLWBytes;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tiles = (M + kBM - 1) / kBM;
    const int my_tiles = (int)blockIdx.x < n_tiles ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (threadIdx.x == 0) {
        for (int k = 0; k < kLStages; ++k) {
            mbar_init(smem_u32(&full[k]), 1);
            mbar_init(smem_u32(&empty[k]), 1);
            if (FIRST) mbar_init(smem_u32(&ready[k]), conv_warps(MODE));  // one arrival per converter warp
        }
        mbar_init(smem_u32(&wbar), 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&accf[b]), 1);
            mbar_init(smem_u32(&acce[b]), epi_warps());  // one arrival per epilogue warp
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed = issued = consumed = committed = 0;
    }
    for (int c = threadIdx.x; c < kHid; c += blockDim.x) {
        s_bias[c] = bias[c];
        if (SELECT) s_w4[c] = sel.w4[c];
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_slot)), "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    volatile int *vfailed = &failed;

    if (warp == 0 && lane == 0) {
        // producer: W once, then the A slices of every tile of this CTA
        const uint32_t wb = smem_u32(&wbar);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(wb), "r"(kLWBytes) : "memory");
        for (int k = 0; k < kLSlices; ++k) tma_load_2d(wbase + k * kLWSlice, &tmW, k * kBK, 0, wb);
        int g = 0;
        // the first configuration row of each tile (kLayerFirst), loaded a tile ahead
        int arow = 0, arow_next = 0;
        if (FIRST && my_tiles > 0) arow = __ldg(&tile_info[blockIdx.x].x);
        for (int j = 0; j < my_tiles && !*vfailed; ++j) {
            const int t = (int)blockIdx.x + j * (int)gridDim.x;
            if (FIRST && j + 1 < my_tiles) arow_next = __ldg(&tile_info[t + (int)gridDim.x].x);
            const int m0 = FIRST ? arow : t * kBM;
            int k = 0;
            for (; k < kLSlices; ++k, ++g) {
                const int st = g % kLStages;
                if (g >= kLStages && !mbar_wait(smem_u32(&empty[st]), ((g / kLStages) - 1) & 1)) {
                    *vfailed = 1;
                    break;
                }
                const uint32_t bar = smem_u32(&full[st]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kLABytes)
                             : "memory");
                tma_load_2d(abase + st * kLABytes, &tmA, k * kBK, m0, bar);
            }
            if (k < kLSlices) break;
            arow = arow_next;
        }
        issued = g;
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_bf16(kBM, kHid);
        bool ok = mbar_wait(smem_u32(&wbar), 0);
        int g = 0, j = 0;
        for (; ok && j < my_tiles && !*vfailed; ++j) {
            const int b = j & 1, u = j >> 1;
            if (u >= 1 && !mbar_wait(smem_u32(&acce[b]), (u - 1) & 1)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t acc = tmem + (uint32_t)(b * kHid);
            for (int k = 0; k < kLSlices; ++k, ++g) {
                const int st = g % kLStages;
                // kLayerFirst: the converters have finished the slice
                if (!mbar_wait(smem_u32(FIRST ? &ready[st] : &full[st]), (g / kLStages) & 1)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a = abase + st * kLABytes, w = wbase + k * kLWSlice;
#pragma unroll
                for (int q = 0; q < kBK / 16; ++q) {
                    const uint64_t ad = smem_desc_sw128(a + 32 * q), bd = smem_desc_sw128(w + 32 * q);
                    const uint32_t accum = (k > 0 || q > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                        ::"r"(acc), "l"(ad), "l"(bd), "r"(idesc), "r"(accum) : "memory");
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(smem_u32(&empty[st])) : "memory");
            }
            if (!ok) break;
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"(smem_u32(&accf[b])) : "memory");
        }
        if (!ok) *vfailed = 1;
        consumed = g;
        committed = j;  // tiles whose accumulator commit was issued
    } else if (FIRST && warp >= 2 + epi_warps()) {
        // converters: warp cw owns rows 16cw .. 16cw+15 of every slice; a pass
        // covers four rows, lane l the 16-byte unit l%8 (physical position) of
        // row l/8 of the pass, so every 8-lane phase touches one 128-byte row
        const int cw = warp - 2 - epi_warps(), ct = (int)threadIdx.x - 32 * (2 + epi_warps());
        // lane l converts logical unit u = l % 8 (columns 8u .. 8u + 7 of the
        // slice) of row l / 8 of each pass; the 128-byte swizzle puts unit u of
        // row r at position u ^ (r % 8), so a phase of eight lanes still covers
        // one whole 128-byte row
        const int uu = lane & 7, rr = lane >> 3;
        const int p0 = uu ^ rr, p1 = uu ^ (rr + 4);  // positions in even and odd passes
        uint8_t *const ring = smem_raw + (abase - smem_u32(smem_raw));  // generic address of the A ring

        float4 bnext = make_float4(0.f, 0.f, 0.f, 0.f);
        if (my_tiles > 0 && ct < kHid / 4) bnext = __ldg(&b_inv[(int64_t)__ldg(&tile_info[blockIdx.x].y) * (kHid / 4) + ct]);
        int g = 0;
        bool ok = true;
        for (int j = 0; j < my_tiles; ++j) {
            const int t = (int)blockIdx.x + j * (int)gridDim.x;
            uint2 *sb = s_binv[j & 1];
            if (ct < kHid / 4) {
                const __nv_bfloat162 lo = __floats2bfloat162_rn(bnext.x, bnext.y);
                const __nv_bfloat162 hi = __floats2bfloat162_rn(bnext.z, bnext.w);
                sb[ct] = make_uint2(*reinterpret_cast<const uint32_t *>(&lo), *reinterpret_cast<const uint32_t *>(&hi));
            }
            if (j + 1 < my_tiles && ct < kHid / 4)
                bnext = __ldg(&b_inv[(int64_t)__ldg(&tile_info[t + (int)gridDim.x].y) * (kHid / 4) + ct]);
            // every converter warp agrees to go on (and has finished the tile
            // before last, whose buffer of the invocation part is rewritten above)
            int all_ok;
            asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n"
                         " bar.red.and.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
                         : "=r"(all_ok) : "r"((unsigned)ok), "n"(kConvBarrier), "n"(32 * conv_warps(MODE)));
            if (!all_ok) break;
            for (int k = 0; k < kLSlices; ++k, ++g) {
                const int st = g % kLStages;
                if (!warp_wait(smem_u32(&full[st]), (g / kLStages) & 1)) {
                    ok = false;
                    break;
                }
                const uint4 bu = reinterpret_cast<const uint4 *>(sb)[8 * k + uu];
                uint8_t *const rows = ring + st * kLABytes + (16 * cw + rr) * 128;
                uint4 v[kConvPasses];
#pragma unroll
                for (int pass = 0; pass < kConvPasses; ++pass)
                    v[pass] = *reinterpret_cast<const uint4 *>(rows + pass * 4 * 128 + ((pass & 1) ? p1 : p0) * 16);
#pragma unroll
                for (int pass = 0; pass < kConvPasses; ++pass)
                    *reinterpret_cast<uint4 *>(rows + pass * 4 * 128 + ((pass & 1) ? p1 : p0) * 16) =
                        relu_add_unit(v[pass], bu);
                // the generic-proxy writes become visible to the tensor cores
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&ready[st])) : "memory");
            }
        }
        if (!ok && lane == 0) *vfailed = 1;
    } else if (warp >= 2) {
        // epilogue: this warp's quarter of every tile's rows, its share of the columns
        constexpr int kCols = kHid * 4 / epi_warps();
        const int quad = warp & 3, half = (warp - 2) >> 2, cbeg = half * kCols;
        const auto row_of = [&](int jj) { return ((int)blockIdx.x + jj * (int)gridDim.x) * kBM + quad * 32 + lane; };
        // kLayerFirst: this warp's staging block (32 rows of 64 bytes, 64-byte swizzle)
        const uint32_t stage = abase + kLStages * kLABytes + (uint32_t)(warp - 2) * kLStageBytes;
        uint8_t *const stage_g = smem_raw + (stage - smem_u32(smem_raw));
        const bool selector = SELECT && half == 0;
        const float b4 = SELECT ? *sel.b4 : 0.f;
        // the selection records of a tile's rows are loaded one tile ahead
        int4 ps = make_int4(0, 0, 0, 0);
        int64_t pcost = 0;
        if (selector && my_tiles > 0 && row_of(0) < M) {
            ps = __ldg(sel.pair_sel + row_of(0));
            pcost = __ldg(sel.pair_cost + row_of(0));
        }
        for (int j = 0; j < my_tiles; ++j) {
            const int b = j & 1, u = j >> 1;
            int4 ps_next = make_int4(0, 0, 0, 0);
            int64_t pcost_next = 0;
            if (selector && j + 1 < my_tiles && row_of(j + 1) < M) {
                ps_next = __ldg(sel.pair_sel + row_of(j + 1));
                pcost_next = __ldg(sel.pair_cost + row_of(j + 1));
            }
            // every epilogue warp agrees on the outcome of the wait (the named
            // barriers below need all of them, or none)
            const bool got = warp_wait(smem_u32(&accf[b]), u & 1);
            if (SELECT) {
                int all_ok;
                asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n"
                             " bar.red.and.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
                             : "=r"(all_ok) : "r"((unsigned)got), "n"(kEpiBarrier), "n"(32 * epi_warps()));
                if (!all_ok) {
                    if (lane == 0) *vfailed = 1;
                    break;
                }
            } else if (!got) {
                if (lane == 0) *vfailed = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int row = row_of(j);
            const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * kHid);
            float dot = 0.f;
#pragma unroll 1
            for (int c0 = cbeg; c0 < cbeg + kCols; c0 += 32) {
                uint32_t r[32];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                      "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                      "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                    : "r"(tbase + (uint32_t)c0));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (SELECT && row >= M) continue;  // (kLayerFirst: M is a whole number of tiles)
                uint32_t pk[16];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float v[16];
                    const float4 *bb = reinterpret_cast<const float4 *>(s_bias + c0 + 16 * h);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 t = bb[q];
                        v[4 * q + 0] = fmaxf(__uint_as_float(r[16 * h + 4 * q + 0]) + t.x, 0.f);
                        v[4 * q + 1] = fmaxf(__uint_as_float(r[16 * h + 4 * q + 1]) + t.y, 0.f);
                        v[4 * q + 2] = fmaxf(__uint_as_float(r[16 * h + 4 * q + 2]) + t.z, 0.f);
                        v[4 * q + 3] = fmaxf(__uint_as_float(r[16 * h + 4 * q + 3]) + t.w, 0.f);
                    }
                    if (SELECT) {
                        const float4 *ww = reinterpret_cast<const float4 *>(s_w4 + c0 + 16 * h);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float4 t = ww[q];
                            dot = fmaf(v[4 * q + 0], t.x, dot);
                            dot = fmaf(v[4 * q + 1], t.y, dot);
                            dot = fmaf(v[4 * q + 2], t.z, dot);
                            dot = fmaf(v[4 * q + 3], t.w, dot);
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
                            pk[8 * h + q] = *reinterpret_cast<const uint32_t *>(&b2);
                        }
                    }
                }
                if (FIRST) {
                    // the staging block is free once the last store from it has read it
                    if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                    __syncwarp();
                    uint4 *srow = reinterpret_cast<uint4 *>(stage_g + lane * 64);
                    const int sw = (lane >> 1) & 3;  // 64-byte swizzle: unit c of row r at c ^ ((r / 2) % 4)
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        srow[c ^ sw] = make_uint4(pk[4 * c], pk[4 * c + 1], pk[4 * c + 2], pk[4 * c + 3]);
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) {
                        asm volatile(
                            "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];"
                            ::"l"(reinterpret_cast<uint64_t>(&tmC)), "r"(c0), "r"(row - lane), "r"(stage) : "memory");
                        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                    }
                }
            }
            // the accumulator is read: the MMAs of tile j + 2 may overwrite it
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce[b])) : "memory");
            if (SELECT) {
                // second halves hand their partial sums to the first halves; the
                // barrier at the top of the next tile orders this read before the
                // next write
                if (half == 1) half_dot[quad * 32 + lane] = dot;
                asm volatile("bar.sync %0, %1;" ::"n"(kEpiBarrier), "n"(32 * epi_warps()) : "memory");
                if (selector && row < M && ps.x >= 0)  // padding rows have no invocation
                    select_row(sel, row, dot + half_dot[quad * 32 + lane] + b4, ps, pcost);
                ps = ps_next;
                pcost = pcost_next;
            }
        }
        // the output stores are complete before the CTA (and its shared memory) ends
        if (FIRST && lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (failed && threadIdx.x == 0) {
        atomicOr(err, 1);
        // let every copy and MMA in flight finish before the shared and tensor
        // memory go away: W, the A slices issued but not consumed, and the
        // accumulators committed (their commits cover every MMA issued before)
        mbar_wait(smem_u32(&wbar), 0);
        for (int g = consumed; g < issued; ++g) mbar_wait(smem_u32(&full[g % kLStages]), (g / kLStages) & 1);
        for (int j = (committed >= 2 ? committed - 2 : 0); j < committed; ++j)
            mbar_wait(smem_u32(&accf[j & 1]), (j >> 1) & 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    });
    return fn;
}

// Row-major BF16 matrix [rows x cols] (cols a multiple of 64), tiles of
// box_rows x 64 with the 128-byte swizzle.
int make_map(CUtensorMap *map, const void *ptr, int64_t rows, int64_t cols, int box_rows) {
    EncodeTiled enc = encoder();
    if (!enc) return LLAMA_ECUDA;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? LLAMA_OK : LLAMA_EINVAL;
}

// Output map of kLayerFirst: row-major BF16 [rows x cols], 32 x 32 blocks,
// 64-byte swizzle (the staging layout of the epilogue).
int make_store_map(CUtensorMap *map, const void *ptr, int64_t rows, int64_t cols) {
    EncodeTiled enc = encoder();
    if (!enc) return LLAMA_ECUDA;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {32, 32};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                           CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? LLAMA_OK : LLAMA_EINVAL;
}

template <int BN>
cudaError_t launch_gemm(const CUtensorMap &ta, const CUtensorMap &tb, int64_t M, int N, int K, const float *bias,
                        int flags, void *c16, float *c32, int ldc, int *err, cudaStream_t s, int splits = 1) {
    constexpr int smem = kStages * (kBM + BN) * kBK * 2 + 1024;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(k_gemm_bf16<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    });
    if (attr != cudaSuccess) return attr;
    const dim3 grid((unsigned)((M + kBM - 1) / kBM), (unsigned)(N / BN), (unsigned)splits);
    k_gemm_bf16<BN><<<grid, kThreads, smem, s>>>(ta, tb, (int)M, N, K, bias, flags,
                                                  static_cast<__nv_bfloat16 *>(c16), c32, ldc, err);
    return cudaGetLastError();
}

int *error_word() {
    static int *w = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        if (cudaMalloc(&w, sizeof(int)) != cudaSuccess) w = nullptr;
        else cudaMemset(w, 0, sizeof(int));
    });
    return w;
}

// C = A . B^T for row-major BF16 operands (see llama_gemm_bf16), enqueued on s.
int gemm(const void *a, const void *b, const float *bias, void *c16, float *c32, int64_t m, int n, int k,
         int flags, cudaStream_t s) {
    if (!a || !b || (!c16 && !c32)) return LLAMA_EINVAL;
    if (m < 1 || m > (1 << 30) || k < kBK || k % kBK || k > (1 << 24)) return LLAMA_EINVAL;
    if (n != 64 && n % 128) return LLAMA_EINVAL;
    if ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15) return LLAMA_EINVAL;
    if ((reinterpret_cast<uintptr_t>(c16) | reinterpret_cast<uintptr_t>(c32)) & 15) return LLAMA_EINVAL;
    int *err = error_word();
    if (!err) return LLAMA_ENOMEM;
    // 256 columns per tile, unless that leaves SMs without a tile: then 128
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LLAMA_ECUDA;
    const int64_t row_tiles = (m + kBM - 1) / kBM;
    const int bn = n == 64 ? 64 : n % 256 == 0 && row_tiles * (n / 256) >= sms ? 256 : 128;
    CUtensorMap ta, tb;
    if (make_map(&ta, a, m, k, kBM) != LLAMA_OK || make_map(&tb, b, n, k, bn) != LLAMA_OK) return LLAMA_EINVAL;
    cudaError_t e;
    if (bn == 64) e = launch_gemm<64>(ta, tb, m, n, k, bias, flags, c16, c32, n, err, s);
    else if (bn == 128) e = launch_gemm<128>(ta, tb, m, n, k, bias, flags, c16, c32, n, err, s);
    else e = launch_gemm<256>(ta, tb, m, n, k, bias, flags, c16, c32, n, err, s);
    return e == cudaSuccess ? LLAMA_OK : LLAMA_ECUDA;
}

namespace {

__device__ __forceinline__ void add4(float4 &a, const float4 &v) {
    a.x += v.x;
    a.y += v.y;
    a.z += v.z;
    a.w += v.w;
}

// c[i] = sum over z < splits of part[z * count + i], added in order of z;
// eight partials' loads in flight at a time.
__global__ void k_sum_splits(const float4 *__restrict__ part, int64_t count4, int splits, float4 *__restrict__ c) {
    constexpr int kBatch = 8;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count4;
         i += (int64_t)gridDim.x * blockDim.x) {
        float4 acc = part[i];
        int z = 1;
        for (; z + kBatch <= splits; z += kBatch) {
            float4 v[kBatch];
#pragma unroll
            for (int j = 0; j < kBatch; ++j) v[j] = part[(z + j) * count4 + i];
#pragma unroll
            for (int j = 0; j < kBatch; ++j) add4(acc, v[j]);
        }
        for (; z < splits; ++z) add4(acc, part[z * count4 + i]);
        c[i] = acc;
    }
}

}  // namespace

int splits_for(int64_t m, int n, int k, int sms) {
    const int64_t tiles = ((m + kBM - 1) / kBM) * (n == 64 ? 1 : n / 128);
    int splits = 1;
    // double the splits while the grid stays within one CTA per SM and every
    // split keeps at least kMinSplitBlocks K blocks
    while (tiles * splits * 2 <= sms && (k / kBK) % (splits * 2) == 0 && k / kBK / (splits * 2) >= kMinSplitBlocks)
        splits *= 2;
    return splits;
}

int gemm_split_k(const void *a, const void *b, float *c32, int64_t m, int n, int k, int splits, float *part,
                 size_t part_bytes, cudaStream_t s) {
    if (!a || !b || !c32 || !part || splits < 1) return LLAMA_EINVAL;
    if (m < 1 || m > (1 << 30) || k < kBK || k % kBK || k > (1 << 24)) return LLAMA_EINVAL;
    if (n != 64 && n % 128) return LLAMA_EINVAL;
    if ((k / kBK) % splits || (size_t)splits * (size_t)m * (size_t)n * sizeof(float) > part_bytes) return LLAMA_EINVAL;
    if ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(c32) |
         reinterpret_cast<uintptr_t>(part)) & 15)
        return LLAMA_EINVAL;
    if (splits == 1) return gemm(a, b, nullptr, nullptr, c32, m, n, k, 0, s);
    int *err = error_word();
    if (!err) return LLAMA_ENOMEM;
    const int bn = n == 64 ? 64 : 128;
    CUtensorMap ta, tb;
    if (make_map(&ta, a, m, k, kBM) != LLAMA_OK || make_map(&tb, b, n, k, bn) != LLAMA_OK) return LLAMA_EINVAL;
    const cudaError_t e = bn == 64 ? launch_gemm<64>(ta, tb, m, n, k, nullptr, 0, nullptr, part, n, err, s, splits)
                                   : launch_gemm<128>(ta, tb, m, n, k, nullptr, 0, nullptr, part, n, err, s, splits);
    if (e != cudaSuccess) return LLAMA_ECUDA;
    const int64_t count4 = m * n / 4;  // n is a multiple of 64
    k_sum_splits<<<(unsigned)std::min<int64_t>((count4 + 255) / 256, 1024), 256, 0, s>>>(
        reinterpret_cast<const float4 *>(part), count4, splits, reinterpret_cast<float4 *>(c32));
    return cudaGetLastError() == cudaSuccess ? LLAMA_OK : LLAMA_ECUDA;
}

// The persistent pair layer (see k_mlp_layer) over m rows: a, BF16 with 256
// columns, holds the rows of A (a_rows of them: m, or the configurations for
// kLayerFirst); w [256 x 256] BF16 (row n = output n), bias [256] FP32; c16
// [m x 256] BF16 out (kLayerFirst) or the fused last layer and selection
// (kLayerSelect).
template <int MODE>
int mlp_layer_impl(const void *a, int64_t a_rows, const void *w, const float *bias, void *c16, int64_t m,
                   const SelectArgs &sel, const int2 *tile_info, const float *b_inv, cudaStream_t s) {
    if (!a || !w || !bias || (MODE != kLayerSelect && !c16) || m < 1 || m > (1 << 30) || a_rows < 1 ||
        a_rows > (1 << 30))
        return LLAMA_EINVAL;
    if (MODE == kLayerFirst && (!tile_info || !b_inv || m % kBM)) return LLAMA_EINVAL;
    if ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(w) | reinterpret_cast<uintptr_t>(c16) |
         reinterpret_cast<uintptr_t>(b_inv)) & 15)
        return LLAMA_EINVAL;
    int *err = error_word();
    if (!err) return LLAMA_ENOMEM;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(k_mlp_layer<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, layer_smem(MODE));
    });
    if (attr != cudaSuccess) return LLAMA_ECUDA;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LLAMA_ECUDA;
    CUtensorMap ta, tw, tc;
    if (make_map(&ta, a, a_rows, kHid, kBM) != LLAMA_OK || make_map(&tw, w, kHid, kHid, kHid) != LLAMA_OK)
        return LLAMA_EINVAL;
    if (MODE == kLayerFirst) {
        if (make_store_map(&tc, c16, m, kHid) != LLAMA_OK) return LLAMA_EINVAL;
    } else {
        tc = ta;  // unused
    }
    const int64_t tiles = (m + kBM - 1) / kBM;
    const unsigned grid = (unsigned)std::min<int64_t>(tiles, sms);
    k_mlp_layer<MODE><<<grid, layer_threads(MODE), layer_smem(MODE), s>>>(
        ta, tw, tc, (int)m, bias, static_cast<__nv_bfloat16 *>(c16), err, sel, tile_info,
        reinterpret_cast<const float4 *>(b_inv));
    return cudaGetLastError() == cudaSuccess ? LLAMA_OK : LLAMA_ECUDA;
}

int mlp_layer_first(const void *a_cfg, int64_t n_cfg, const float *b_inv, const int2 *tile_info, const void *w,
                    const float *bias, void *c16, int64_t m, cudaStream_t s) {
    return mlp_layer_impl<kLayerFirst>(a_cfg, n_cfg, w, bias, c16, m, SelectArgs{}, tile_info, b_inv, s);
}

int mlp_layer_select(const void *a, const void *w, const float *bias, int64_t m, const SelectArgs &sel,
                     cudaStream_t s) {
    return mlp_layer_impl<kLayerSelect>(a, m, w, bias, nullptr, m, sel, nullptr, nullptr, s);
}

}  // namespace sgk

using namespace sgk;

extern "C" int llama_gemm_bf16(const void *a, const void *b, const float *bias, void *c_bf16, float *c_f32,
                               int64_t m, int32_t n, int32_t k, int32_t flags, void *stream) {
    return gemm(a, b, bias, c_bf16, c_f32, m, n, k, flags, static_cast<cudaStream_t>(stream));
}

extern "C" int llama_gemm_error(int32_t clear) {
    int *err = error_word();
    if (!err) return LLAMA_ENOMEM;
    int h = 0;
    if (cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return LLAMA_ECUDA;
    if (clear && h) cudaMemset(err, 0, sizeof(int));
    return h ? LLAMA_ETIMEOUT : LLAMA_OK;
}
