// mlp_gemm.cu -- BF16 GEMM on the 5th-generation tensor cores (tcgen05),
// for the dense layers of the MLP energy surrogate.
//
// C[M x N] (FP32) = A[M x K] . B[N x K]^T, A and B row-major BF16 (both
// "K-major").  Persistent kernel, one CTA per SM, in clusters of two CTAs
// that compute the 128 x 256 output tiles of two adjacent row blocks in the
// same column block, so that the 256 x 64 B tile of each k-step is read from
// L2 once per cluster instead of once per CTA.  Six warps with fixed roles:
//   * one thread of warp 0 streams the CTA's 128 x 64 tile of A and its half
//     (128 x 64) of the shared B tile with TMA (cp.async.bulk.tensor, 128-byte
//     swizzle, out-of-range rows and columns zero-filled), the B half
//     multicast into both CTAs' stage, into a ring of kStages shared-memory
//     stages, each completing a transaction-count mbarrier; a stage is
//     refilled once the products of both CTAs have read it;
//   * one thread of warp 1 issues four tcgen05.mma (M 128, N 256, K 16) per
//     stage into one of two FP32 accumulators of 256 tensor-memory columns,
//     frees each stage in both CTAs with a multicast tcgen05.commit, and
//     commits the accumulator when a tile's last product is issued;
//   * warps 2..5 drain a finished accumulator with tcgen05.ld (warp w reads
//     tensor-memory lanes 32 (w mod 4) ..), apply the bias and the layer's
//     output transform, store with 16-byte vector stores, and hand the
//     accumulator back -- so the epilogue of one tile runs while the tensor
//     core works on the next.
//
// Every wait on an mbarrier is bounded: after kWaitLimit polls the waiting
// role records PAMD_ETIMEOUT and raises a shared abort flag, the others stop
// at their next wait, the CTA waits (bounded) for its own copies and products
// in flight, meets its partner at a cluster barrier (so that neither leaves
// while the other may still write to it), frees its tensor memory and returns.
// A partner that timed out stops feeding the other, whose own bounded waits
// then run out as well.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "pamd_internal.h"

namespace pamd {

namespace {

constexpr int kBM = 128, kBN = kGemmTileN, kBK = 64, kStages = 4;
// warp 0: TMA producer, warp 1: MMA issuer, warps 2..9: epilogue (two warps
// per tensor-memory lane quarter, each taking one half of the tile's columns)
constexpr int kEpiWarps = 8, kThreads = 64 + 32 * kEpiWarps, kEpiThreads = 32 * kEpiWarps;
constexpr int kTileA = kBM * kBK * 2;  // 16 KiB
constexpr int kTileB = kBN * kBK * 2;  // 32 KiB
constexpr int kStageBytes = kTileA + kTileB;
constexpr int kTmemCols = 2 * kBN;     // two accumulators: all 512 columns
constexpr uint32_t kWaitLimit = 1u << 22;

// instruction descriptor of tcgen05.mma.kind::f16: D FP32 (bits 4-5 = 1),
// A BF16 (bits 7-9 = 1), B BF16 (bits 10-12 = 1), both K-major, N >> 3 at
// bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: K-major operand in the 128-byte swizzle
// layout, 8-row groups 1024 bytes apart (stride byte offset), descriptor
// version 1 (bits 46-47), swizzle mode 2 = 128 B (bits 61-63).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait (polls, then polls with a short sleep); false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t i = 0; i < kWaitLimit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i >= 1024) __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// TMA: tile of a 2-D tensor map at element coordinates (x = column, y = row)
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem), "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

// TMA load multicast to the CTAs of the cluster in `mask`: the tile lands at
// the same shared-memory offset in each and completes each one's mbarrier at
// the same offset
__device__ __forceinline__ void tma_load_2d_mc(uint32_t dst, const CUtensorMap* map, int x, int y,
                                               uint32_t bar, uint16_t mask) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        ".multicast::cluster [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar), "h"(mask)
        : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                     : "memory");
}

// arrive on the mbarrier at this offset in every CTA of `mask` once the
// products issued so far are done
__device__ __forceinline__ void mma_commit_mc(uint32_t bar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            bar),
        "h"(mask)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 32 columns of FP32 accumulator for this thread's row (TMEM lane)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}


__device__ __forceinline__ float sigmoid(float z) { return __fdividef(1.0f, 1.0f + __expf(-z)); }

// 32 consecutive FP32 values of one row: vector stores when the whole chunk
// is inside the matrix and 16-byte aligned, else element by element
__device__ __forceinline__ void store_row32(float* dst, const float (&v)[32], int n, bool vec) {
    if (vec && n == 32) {
        float4* d = reinterpret_cast<float4*>(dst);
#pragma unroll
        for (int q = 0; q < 8; ++q) d[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (j < n) dst[j] = v[j];
    }
}

__device__ __forceinline__ void store_row32_bf16(__nv_bfloat16* dst, const float (&v)[32], int n,
                                                 bool vec) {
    if (vec && n == 32) {
        uint4* d = reinterpret_cast<uint4*>(dst);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t w[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const __nv_bfloat162 h = __floats2bfloat162_rn(v[8 * q + 2 * t], v[8 * q + 2 * t + 1]);
                w[t] = *reinterpret_cast<const uint32_t*>(&h);
            }
            d[q] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (j < n) dst[j] = __float2bfloat16(v[j]);
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Epilogue of one half (128 columns) of a 128 x 256 tile: accumulator
// columns of this warp's 32 tensor-memory lanes (rows m0 + 32q + lane);
// taddr and n0 point at the half's first column.
__device__ __forceinline__ void epilogue_tile(const GemmArgs& g, uint32_t taddr, int row, int n0,
                                              int ntile, int ntiles, int half) {
    const bool row_ok = row < g.M;
    float head = 0.0f;
    __nv_bfloat16* Cb = static_cast<__nv_bfloat16*>(g.Cb);
    __nv_bfloat16* CbT = static_cast<__nv_bfloat16*>(g.CbT);
    const bool vf = (g.vec_ok & 1) != 0, vb = (g.vec_ok & 2) != 0;
#pragma unroll 1
    for (int cc = 0; cc < kBN / 64; ++cc) {
        float v[32];
        tmem_ld32(taddr + (uint32_t)(cc * 32), v);
        const int col0 = n0 + cc * 32;
        const int n = min(32, g.N - col0);
        if (!row_ok || n <= 0) continue;
        if (g.bias) {
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] += (j < n) ? g.bias[col0 + j] : 0.0f;
        }
        const size_t o = (size_t)row * g.ldc + col0;
        if (g.C) store_row32(g.C + o, v, n, vf);
        if (g.epi == kEpiSilu || g.epi == kEpiHead) {
            float ds[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float sg = sigmoid(v[j]);
                ds[j] = sg * (1.0f + v[j] * (1.0f - sg));
                v[j] *= sg;  // silu
            }
            if (g.Cs) store_row32(g.Cs + o, ds, n, vf);
            if (g.epi == kEpiHead) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float w = (j < n) ? g.vec[col0 + j] : 0.0f;
                    head = fmaf(w, v[j], head);
                    v[j] = w * ds[j];
                }
            }
        } else if (g.epi == kEpiMul) {
            const float* mr = g.mul + o;
            if (vf && n == 32) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float4 t = reinterpret_cast<const float4*>(mr)[q];
                    v[4 * q] *= t.x;
                    v[4 * q + 1] *= t.y;
                    v[4 * q + 2] *= t.z;
                    v[4 * q + 3] *= t.w;
                }
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] *= (j < n) ? mr[j] : 0.0f;
            }
        }
        if (Cb) store_row32_bf16(Cb + (size_t)row * g.ldcb + col0, v, n, vb);
        if (CbT) {
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (j < n) CbT[(size_t)(col0 + j) * g.ldt + row] = __float2bfloat16(v[j]);
        }
    }
    if (g.epi == kEpiHead && row_ok)
        g.part[(size_t)row * (kGemmHeadParts * ntiles) + kGemmHeadParts * ntile + half] = head;
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    gemm_bf16_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                const __grid_constant__ CUtensorMap tmB,
                                                                const __grid_constant__ GemmArgs g) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long full_bar[kStages], empty_bar[kStages];
    __shared__ __align__(8) unsigned long long accf_bar[2], acce_bar[2], done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_abort, s_issued, s_consumed;
    // 1024-byte aligned stages: [A0 | B0 | A1 | B1 | ...]
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // The two CTAs of a cluster take row blocks 2p and 2p + 1 of the same
    // column block: each loads its A tile and half of the shared B tile,
    // multicast to both.
    const int MT = (g.M + kBM - 1) / kBM, NT = (g.N + kBN - 1) / kBN;
    const int tiles = ((MT + 1) / 2) * NT;  // tile pairs
    const int KB = (g.K + kBK - 1) / kBK;
    const int crank = (int)cluster_rank();
    const int cid = blockIdx.x >> 1, ncl = gridDim.x >> 1;

    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"((uint32_t)kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) {
            mbar_init(smem_u32(&full_bar[st]), 1);
            mbar_init(smem_u32(&empty_bar[st]), 2);  // both CTAs' products have read it
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(smem_u32(&accf_bar[q]), 1);
            mbar_init(smem_u32(&acce_bar[q]), kEpiThreads);
        }
        mbar_init(smem_u32(&done_bar), 1);
        s_abort = 0;
        s_issued = 0;
        s_consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    cluster_sync();  // the peer's barriers exist before any multicast reaches them
    const uint32_t tmem = tmem_slot;
    volatile int* abort_flag = &s_abort;

    if (warp == 0) {
        if (lane == 0) {  // TMA producer
            long long gk = 0;
            bool stop = false;
            for (int t = cid; t < tiles && !stop; t += ncl) {
                // A box of an odd last row block's missing partner, or a B half
                // past column N, would lie wholly outside its matrix: read a
                // valid box instead (its products land in rows / columns the
                // epilogue drops)
                const int n0 = (t % NT) * kBN;
                const int ya = min((2 * (t / NT) + crank) * kBM, (MT - 1) * kBM);
                const int yb = (n0 + crank * (kBN / 2) < g.N) ? n0 + crank * (kBN / 2) : n0;
                for (int kb = 0; kb < KB; ++kb, ++gk) {
                    const int st = (int)(gk % kStages);
                    if (gk >= kStages &&
                        !mbar_wait(smem_u32(&empty_bar[st]), (uint32_t)((gk / kStages - 1) & 1))) {
                        *abort_flag = 1;
                    }
                    if (*abort_flag) {
                        stop = true;
                        break;
                    }
                    const uint32_t fb = smem_u32(&full_bar[st]);
                    const uint32_t ta = base + (uint32_t)(st * kStageBytes);
                    mbar_expect_tx(fb, (uint32_t)kStageBytes);
                    tma_load_2d(ta, &tmA, kb * kBK, ya, fb);
                    tma_load_2d_mc(ta + kTileA + crank * (kTileB / 2), &tmB, kb * kBK, yb, fb,
                                   (uint16_t)0x3);
                }
            }
            s_issued = (int)gk;
            // the peer's last releases of this CTA's stages land before it exits
            for (long long u = gk > kStages ? gk - kStages : 0; u < gk && !*abort_flag; ++u)
                if (!mbar_wait(smem_u32(&empty_bar[u % kStages]), (uint32_t)((u / kStages) & 1)))
                    *abort_flag = 1;
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            long long gk = 0;
            int i = 0;
            bool stop = false;
            for (int t = cid; t < tiles && !stop; t += ncl, ++i) {
                const int acc = i & 1;
                if (i >= 2 && !mbar_wait(smem_u32(&acce_bar[acc]), (uint32_t)((i / 2 - 1) & 1))) {
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t td = tmem + (uint32_t)(acc * kBN);
                for (int kb = 0; kb < KB; ++kb, ++gk) {
                    const int st = (int)(gk % kStages);
                    if (!mbar_wait(smem_u32(&full_bar[st]), (uint32_t)((gk / kStages) & 1))) *abort_flag = 1;
                    if (*abort_flag) {
                        stop = true;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t ta = base + (uint32_t)(st * kStageBytes);
#pragma unroll
                    for (int k = 0; k < kBK / 16; ++k)
                        mma_bf16(td, sw128_desc(ta + k * 32), sw128_desc(ta + kTileA + k * 32),
                                 (kb > 0 || k > 0) ? 1u : 0u);
                    mma_commit_mc(smem_u32(&empty_bar[st]), (uint16_t)0x3);
                }
                if (!stop) mma_commit(smem_u32(&accf_bar[acc]));
            }
            s_consumed = (int)gk;
            // tracks every product issued before it, also on the abort path
            mma_commit(smem_u32(&done_bar));
        }
    } else {  // epilogue warps 2..9
        const int q = warp & 3;  // tensor-memory lane quarter this warp may access
        const int half = (warp - 2) >> 2;
        int i = 0;
        for (int t = cid; t < tiles; t += ncl, ++i) {
            const int acc = i & 1;
            if (!mbar_wait(smem_u32(&accf_bar[acc]), (uint32_t)((i / 2) & 1))) *abort_flag = 1;
            __syncwarp();
            if (*abort_flag) break;
            tc_fence_after();
            const int m0 = (2 * (t / NT) + crank) * kBM, nt = t % NT;
            const uint32_t taddr =
                tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * kBN + half * (kBN / 2));
            epilogue_tile(g, taddr, m0 + q * 32 + lane, nt * kBN + half * (kBN / 2), nt, NT, half);
            tc_fence_before();
            mbar_arrive(smem_u32(&acce_bar[acc]));
        }
    }
    __syncwarp();
    __syncthreads();
    if (tid == 0) {
        if (*abort_flag) {
            atomicCAS(g.status, 0, PAMD_ETIMEOUT);
            // copies issued but never consumed must land before the CTA exits
            for (long long gk = s_consumed; gk < s_issued; ++gk)
                mbar_wait(smem_u32(&full_bar[gk % kStages]), (uint32_t)((gk / kStages) & 1));
        }
        mbar_wait(smem_u32(&done_bar), 0u);  // products in flight
    }
    tc_fence_before();
    __syncthreads();
    // neither CTA leaves while the other may still write its shared memory or
    // arrive on its barriers
    cluster_sync();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"((uint32_t)kTmemCols)
                     : "memory");
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// Tensor map of a row-major BF16 matrix [rows][ld] read in box_rows x 64-column
// boxes with the 128-byte swizzle; columns >= cols and rows >= rows read as 0.
bool encode_operand(CUtensorMap* map, const void* ptr, int rows, int cols, int ld, int box_rows) {
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// True when p is device memory of device dev (not host, pinned host, managed
// or another GPU's memory).
bool on_device(const void* p, int dev) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

constexpr int kMaxDevices = 64;

// Kernel attribute and resident cluster count, once per device.
cudaError_t gemm_setup(int dev, int* max_clusters_out) {
    const size_t smem = (size_t)kStages * kStageBytes + 1024;
    static std::once_flag once[kMaxDevices];
    static cudaError_t attr[kMaxDevices];
    static int max_clusters[kMaxDevices];
    std::call_once(once[dev], [&] {
        cudaError_t e = cudaFuncSetAttribute(gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        // persistent grid: as many two-CTA clusters as can be resident at once
        // (an SM left without a partner in its GPC hosts none)
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(2, 1, 1);
        cfg.blockDim = dim3(kThreads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        int mc = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(&mc, gemm_bf16_kernel, &cfg);
        if (e == cudaSuccess && mc < 1) e = cudaErrorInvalidConfiguration;
        attr[dev] = e;
        max_clusters[dev] = mc;
    });
    if (max_clusters_out) *max_clusters_out = max_clusters[dev];
    return attr[dev];
}

cudaError_t gemm_prepare_device() {
    int dev = 0;
    const cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    return gemm_setup(dev, nullptr);
}

cudaError_t launch_gemm_bf16(const GemmArgs& ga, cudaStream_t s) {
    if (ga.M <= 0 || ga.N <= 0 || ga.K <= 0 || (ga.K & 7) || (ga.lda & 7) || (ga.ldb & 7) ||
        (reinterpret_cast<uintptr_t>(ga.A) & 15) || (reinterpret_cast<uintptr_t>(ga.B) & 15))
        return cudaErrorInvalidValue;
    int dev = 0;
    cudaError_t de = cudaGetDevice(&dev);
    if (de != cudaSuccess) return de;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    // The B tile is multicast by TMA into both CTAs of a cluster: the tensor
    // maps must cover this GPU's own memory only.
    if (!on_device(ga.A, dev) || !on_device(ga.B, dev)) return cudaErrorInvalidValue;
    CUtensorMap tmA, tmB;
    if (!encode_operand(&tmA, ga.A, ga.M, ga.K, ga.lda, kBM) ||
        !encode_operand(&tmB, ga.B, ga.N, ga.K, ga.ldb, kBN / 2))
        return cudaErrorInvalidValue;
    GemmArgs g = ga;
    auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    const bool f_ok = (g.ldc % 4 == 0) && al16(g.C) && al16(g.Cs) && al16(g.mul);
    const bool b_ok = (g.ldcb % 8 == 0) && al16(g.Cb);
    g.vec_ok = (f_ok ? 1 : 0) | (b_ok ? 2 : 0);
    const size_t smem = (size_t)kStages * kStageBytes + 1024;
    int max_clusters = 0;
    const cudaError_t se = gemm_setup(dev, &max_clusters);
    if (se != cudaSuccess) return se;
    // one cluster per pair of row blocks and column block, at most max_clusters
    const long long pairs = (long long)((g.M + 2 * kBM - 1) / (2 * kBM)) * ((g.N + kBN - 1) / kBN);
    const int grid = 2 * (int)(pairs < max_clusters ? pairs : max_clusters);
    gemm_bf16_kernel<<<grid, kThreads, smem, s>>>(tmA, tmB, g);
    return cudaGetLastError();
}

}  // namespace pamd

using namespace pamd;

namespace {

int gemm_entry(const void* A, const void* B, float* C, int32_t M, int32_t N, int32_t K, int32_t lda,
               int32_t ldb, int32_t ldc, int32_t reps, void* stream, float* ms_out) {
    if (!A || !B || !C || M < 1 || N < 1 || K < 1 || (K & 7) || (lda & 7) || (ldb & 7) ||
        lda < K || ldb < K || ldc < N || (reinterpret_cast<uintptr_t>(A) & 15) ||
        (reinterpret_cast<uintptr_t>(B) & 15) || reps < 1 || reps > 1000) {
        set_last_error("pamd_gemm_bf16: null pointer, or sizes / leading dimensions invalid "
                       "(K, lda, ldb multiples of 8; A, B 16-byte aligned; reps 1..1000)");
        return PAMD_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        set_last_error("pamd_gemm_bf16: no usable current device");
        return PAMD_ECUDA;
    }
    if (!on_device(A, dev) || !on_device(B, dev)) {
        set_last_error("pamd_gemm_bf16: A and B must be device memory of the current device");
        return PAMD_EINVAL;
    }
    // one status word per device, allocated on that device's first call
    static std::mutex mu;
    static int* status_of[kMaxDevices] = {};
    int* status = nullptr;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!status_of[dev] && cudaMalloc(&status_of[dev], sizeof(int)) != cudaSuccess) {
            status_of[dev] = nullptr;
            cudaGetLastError();
            set_last_error("pamd_gemm_bf16: status word");
            return PAMD_ENOMEM;
        }
        status = status_of[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    GemmArgs g{};
    g.A = A;
    g.B = B;
    g.C = C;
    g.M = M;
    g.N = N;
    g.K = K;
    g.lda = lda;
    g.ldb = ldb;
    g.ldc = ldc;
    g.epi = kEpiStore;
    g.status = status;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);
    if (e == cudaSuccess && ms_out) e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess && ms_out) e = cudaEventCreate(&ev[1]);
    if (e == cudaSuccess && ms_out) e = cudaEventRecord(ev[0], s);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_gemm_bf16(g, s);
    if (e == cudaSuccess && ms_out) e = cudaEventRecord(ev[1], s);
    int st = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && ms_out) {
        float ms = 0.0f;
        e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
        *ms_out = ms / (float)reps;
    }
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    if (e != cudaSuccess) {
        set_last_error(std::string("pamd_gemm_bf16: ") + cudaGetErrorString(e));
        return PAMD_ECUDA;
    }
    if (st) {
        set_last_error("pamd_gemm_bf16: tensor-core pipeline timed out");
        return st;
    }
    return PAMD_OK;
}

}  // namespace

extern "C" int pamd_gemm_bf16(const void* A, const void* B, float* C, int32_t M, int32_t N,
                              int32_t K, int32_t lda, int32_t ldb, int32_t ldc, void* stream) {
    return gemm_entry(A, B, C, M, N, K, lda, ldb, ldc, 1, stream, nullptr);
}

extern "C" int pamd_gemm_bf16_time(const void* A, const void* B, float* C, int32_t M, int32_t N,
                                   int32_t K, int32_t lda, int32_t ldb, int32_t ldc, int32_t reps,
                                   void* stream, float* ms_out) {
    if (!ms_out) {
        set_last_error("pamd_gemm_bf16_time: null ms_out");
        return PAMD_EINVAL;
    }
    return gemm_entry(A, B, C, M, N, K, lda, ldb, ldc, reps, stream, ms_out);
}
