// peak.cu -- FP32 throughput microbenchmark: the denominator of the force
// kernel's roofline.  Every thread runs independent chains of fused
// multiply-adds (no chain waits on another), the grid fills every SM to its
// thread limit, and the launch is timed with CUDA events.  Two forms: scalar
// fma.rn.f32 (FFMA) and packed fma.rn.f32x2 (two lanes per instruction); the
// larger rate is the measured FP32 peak.
#include <cuda_runtime.h>

#include <string>

#include "pamd_internal.h"
#include "../../include/pamd_bench.h"

namespace pamd {
namespace {

constexpr int kChains = 16;       // independent FMA chains per thread (scalar form)
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) ffma_kernel(float* out, int iters, float a, float b) {
    float acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = (float)threadIdx.x * 1e-3f + (float)c;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = fmaf(acc[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

__global__ void __launch_bounds__(kPeakThreads) ffma2_kernel(float* out, int iters, float a, float b) {
    float2 acc[kChains / 2];
    const float2 av = make_float2(a, a), bv = make_float2(b, b);
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c)
        acc[c] = make_float2((float)threadIdx.x * 1e-3f + (float)c, (float)c + 0.5f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains / 2; ++c) acc[c] = __ffma2_rn(acc[c], av, bv);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) s += acc[c].x + acc[c].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace pamd

using namespace pamd;

extern "C" int pamd_fp32_peak(int32_t packed, int32_t iters, int32_t reps, void* stream,
                              float* out_dev, double* tflops, double* ms) {
    if ((packed != 0 && packed != 1) || iters < 1 || iters > (1 << 24) || reps < 1 || reps > 1000 ||
        !out_dev || !tflops) {
        set_last_error("pamd_fp32_peak: packed 0/1, iters 1..2^24, reps 1..1000, out_dev and tflops required");
        return PAMD_EINVAL;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    if (e != cudaSuccess) {
        set_last_error(std::string("pamd_fp32_peak: ") + cudaGetErrorString(e));
        return PAMD_ECUDA;
    }
    const int blocks = sms * (per_sm / kPeakThreads);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    auto launch = [&] {
        if (packed)
            ffma2_kernel<<<blocks, kPeakThreads, 0, s>>>(out_dev, iters, 0.999f, 1e-3f);
        else
            ffma_kernel<<<blocks, kPeakThreads, 0, s>>>(out_dev, iters, 0.999f, 1e-3f);
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        launch();  // warm-up
        e = cudaEventRecord(e0, s);
    }
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        set_last_error(std::string("pamd_fp32_peak: ") + cudaGetErrorString(e));
        return PAMD_ECUDA;
    }
    // kChains fma per thread per iteration, 2 flop each (the packed form runs
    // kChains / 2 instructions of two lanes)
    const double flop = 2.0 * kChains * (double)iters * (double)blocks * kPeakThreads * reps;
    *tflops = flop / (t * 1e-3) / 1e12;
    if (ms) *ms = t;
    return PAMD_OK;
}

extern "C" int32_t pamd_fp32_peak_threads(void) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return sms * (per_sm / pamd::kPeakThreads) * pamd::kPeakThreads;
}
