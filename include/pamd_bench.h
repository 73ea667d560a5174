/*
 * pamd_bench.h -- measurement helpers of libpamd.  The paper has no
 * counterpart: these give the roofline of the force kernel a measured
 * denominator instead of a figure derived from unit counts and clocks.
 */
#ifndef PAMD_BENCH_H
#define PAMD_BENCH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * FP32 fused-multiply-add throughput of the current device.  A grid that
 * fills every SM to its thread limit runs `iters` iterations of 16
 * independent FMA chains per thread, in scalar fma.rn.f32 (packed = 0) or
 * packed fma.rn.f32x2 (packed = 1, two lanes per instruction); one untimed
 * launch, then `reps` launches timed with CUDA events on `stream`.
 * out_dev: device float buffer of pamd_fp32_peak_threads() elements (each
 * thread stores its sum there so the chains are not optimised away).
 * tflops: host output, 2 flop per FMA.  ms: host output (total of the timed
 * launches) or NULL.  iters 1..2^24, reps 1..1000.  Synchronises `stream`.
 * Errors: PAMD_EINVAL, PAMD_ECUDA.
 */
int pamd_fp32_peak(int32_t packed, int32_t iters, int32_t reps, void* stream, float* out_dev,
                   double* tflops, double* ms);

/* Threads (= floats of out_dev) of one pamd_fp32_peak launch on the current
 * device, or 0 without a device. */
int32_t pamd_fp32_peak_threads(void);

#ifdef __cplusplus
}
#endif
#endif /* PAMD_BENCH_H */
