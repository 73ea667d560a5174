// mlp_gemm.cu -- BF16 GEMM on the 5th-generation tensor cores (tcgen05),
// for the dense layers of the MLP energy surrogate.
//
// C[M x N] (FP32) = A[M x K] . B[N x K]^T, A and B row-major BF16 (both
// "K-major").  One CTA computes a 128 x 128 tile: 4 warps copy 128 x 64 tiles
// of A and B into shared memory in the 128-byte-swizzled K-major layout
// (two stages), one thread issues four tcgen05.mma (M 128, N 128, K 16) per
// stage with the accumulator in tensor memory (128 columns of FP32), and a
// tcgen05.commit signals an mbarrier when the stage may be overwritten.  The
// epilogue reads the accumulator with tcgen05.ld (warp w owns rows 32w..32w+31)
// and applies an optional bias and output transform.
//
// Every wait on an mbarrier is bounded: after kWaitLimit polls the kernel
// records PAMD_ETIMEOUT, waits a bounded time more for its own MMAs, frees its
// tensor memory and returns.
#include <cuda_bf16.h>

#include "pamd_internal.h"

namespace pamd {

namespace {

constexpr int kBM = 128, kBN = 128, kBK = 64, kThreads = 128;
constexpr int kTileBytes = kBM * kBK * 2;  // 16 KiB per operand tile
constexpr int kTmemCols = 128;
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

// bounded wait; returns false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t i = 0; i < kWaitLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
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

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void st_shared_zero16(uint32_t dst) {
    asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};" ::"r"(dst), "r"(0u) : "memory");
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

// Copy a 128-row x 64-column BF16 tile (rows r0.., columns k0..) of a
// row-major matrix into the swizzled layout; rows or columns outside the
// matrix are zero.  K (and ld) must be multiples of 8.
__device__ __forceinline__ void load_tile(uint32_t tile, const __nv_bfloat16* __restrict__ X,
                                          int rows, int K, int ld, int r0, int k0) {
    for (int idx = threadIdx.x; idx < kBM * 8; idx += kThreads) {
        const int r = idx >> 3, c = idx & 7;
        const uint32_t dst = tile + (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4));
        const int gr = r0 + r, gk = k0 + c * 8;
        if (gr < rows && gk < K)
            cp_async16(dst, X + (size_t)gr * ld + gk);
        else
            st_shared_zero16(dst);
    }
}

}  // namespace

__device__ __forceinline__ float sigmoid(float z) { return 1.0f / (1.0f + __expf(-z)); }

__global__ void __launch_bounds__(kThreads, 1) gemm_bf16_kernel(const __grid_constant__ GemmArgs g) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ uint32_t tmem_slot;
    // 1024-byte aligned operand tiles: [A0 | B0 | A1 | B1]
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    const uint32_t bar[2] = {smem_u32(&mbar[0]), smem_u32(&mbar[1])};
    const __nv_bfloat16* A = static_cast<const __nv_bfloat16*>(g.A);
    const __nv_bfloat16* B = static_cast<const __nv_bfloat16*>(g.B);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"((uint32_t)kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(bar[0], 1);
        mbar_init(bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    // Mainloop.  Control flow is uniform across the block: every thread sees
    // the same k-block count and the same (block-reduced) timeout flag.
    const int KB = (g.K + kBK - 1) / kBK;
    uint32_t phase[2] = {0u, 0u};
    bool ok = true;
    int committed = 0;
    for (int kb = 0; kb < KB; ++kb) {
        const int s = kb & 1;
        if (kb >= 2) {  // the MMAs of k-block kb-2 have finished reading stage s
            if (!mbar_wait(bar[s], phase[s])) ok = false;
            phase[s] ^= 1u;
        }
        if (!__syncthreads_and(ok)) break;
        const uint32_t ta = base + (uint32_t)(s * 2 * kTileBytes);
        const uint32_t tb = ta + kTileBytes;
        load_tile(ta, A, g.M, g.K, g.lda, m0, kb * kBK);
        load_tile(tb, B, g.N, g.K, g.ldb, n0, kb * kBK);
        asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k)
                mma_bf16(tmem, sw128_desc(ta + k * 32), sw128_desc(tb + k * 32),
                         (kb > 0 || k > 0) ? 1u : 0u);
            mma_commit(bar[s]);
        }
        committed = kb + 1;
    }
    // The last commit tracks every MMA issued before it: wait for it (on the
    // error path too, so that no MMA still writes the tensor memory we free).
    if (committed > 0) {
        const int s = (committed - 1) & 1;
        if (!mbar_wait(bar[s], phase[s])) ok = false;
    }
    ok = __syncthreads_and(ok);
    if (!ok) {
        if (tid == 0) atomicCAS(g.status, 0, PAMD_ETIMEOUT);
    } else {
        tc_fence_after();
        const int row = m0 + warp * 32 + lane;
        const bool row_ok = row < g.M;
        float head = 0.0f;
        __nv_bfloat16* Cb = static_cast<__nv_bfloat16*>(g.Cb);
        __nv_bfloat16* CbT = static_cast<__nv_bfloat16*>(g.CbT);
#pragma unroll 1
        for (int cc = 0; cc < kBN / 32; ++cc) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cc * 32), v);
            if (!row_ok) continue;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int col = n0 + cc * 32 + j;
                if (col >= g.N) continue;
                const float z = v[j] + (g.bias ? g.bias[col] : 0.0f);
                const size_t o = (size_t)row * g.ldc + col;
                if (g.C) g.C[o] = z;
                float out = z;
                if (g.epi == kEpiSilu || g.epi == kEpiHead) {
                    const float sg = sigmoid(z);
                    const float ds = sg * (1.0f + z * (1.0f - sg));
                    if (g.Cs) g.Cs[o] = ds;
                    if (g.epi == kEpiSilu) {
                        out = z * sg;
                    } else {
                        head += g.vec[col] * (z * sg);
                        out = g.vec[col] * ds;
                    }
                } else if (g.epi == kEpiMul) {
                    out = z * g.mul[o];
                }
                const __nv_bfloat16 ob = __float2bfloat16(out);
                if (Cb) Cb[(size_t)row * g.ldcb + col] = ob;
                if (CbT) CbT[(size_t)col * g.ldt + row] = ob;
            }
        }
        if (g.epi == kEpiHead && row_ok) g.part[(size_t)row * gridDim.x + blockIdx.x] = head;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"((uint32_t)kTmemCols)
                     : "memory");
}

cudaError_t launch_gemm_bf16(const GemmArgs& g, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0 || g.K <= 0 || (g.K & 7) || (g.lda & 7) || (g.ldb & 7))
        return cudaErrorInvalidValue;
    const size_t smem = 4 * (size_t)kTileBytes + 1024;
    static bool configured = false;
    if (!configured) {
        const cudaError_t e =
            cudaFuncSetAttribute(gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const dim3 grid((g.N + kBN - 1) / kBN, (g.M + kBM - 1) / kBM);
    gemm_bf16_kernel<<<grid, kThreads, smem, s>>>(g);
    return cudaGetLastError();
}

}  // namespace pamd

using namespace pamd;

extern "C" int pamd_gemm_bf16(const void* A, const void* B, float* C, int32_t M, int32_t N,
                              int32_t K, int32_t lda, int32_t ldb, int32_t ldc, void* stream) {
    if (!A || !B || !C || M < 1 || N < 1 || K < 1 || (K & 7) || (lda & 7) || (ldb & 7) ||
        lda < K || ldb < K || ldc < N || (reinterpret_cast<uintptr_t>(A) & 15) ||
        (reinterpret_cast<uintptr_t>(B) & 15)) {
        set_last_error("pamd_gemm_bf16: null pointer, or sizes / leading dimensions invalid "
                       "(K, lda, ldb multiples of 8; A, B 16-byte aligned)");
        return PAMD_EINVAL;
    }
    static int* status = nullptr;
    if (!status && cudaMalloc(&status, sizeof(int)) != cudaSuccess) {
        set_last_error("pamd_gemm_bf16: status word");
        return PAMD_ENOMEM;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return PAMD_ECUDA;
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
    cudaError_t e = launch_gemm_bf16(g, s);
    int st = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
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
