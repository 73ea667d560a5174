// pamd_device.cuh -- device-side random numbers and deterministic exponential.
#pragma once

#include <stdint.h>

namespace pamd {

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of the
// 4x32 S-P network with multipliers 0xD2511F53 / 0xCD9E8D57, the key bumped
// by the Weyl constants 0x9E3779B9 / 0xBB67AE85 after every round.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint2 seed_key(unsigned long long seed) {
    return make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
}

// Uniform in (0,1) from the top 23 bits: (k + 1/2) 2^-23, exact in binary32.
__device__ __forceinline__ float uniform23(uint32_t u) {
    return (__uint2float_rn(u >> 9) + 0.5f) * 1.1920928955078125e-07f;
}

// Three standard normals by the Box-Muller transform of one Philox block.
__device__ __forceinline__ float3 normal3(unsigned long long seed, uint32_t atom, uint32_t slot,
                                          uint32_t step, uint32_t purpose) {
    const uint4 o = philox4x32_10(make_uint4(atom, slot, step, purpose), seed_key(seed));
    const float r0 = sqrtf(-2.0f * logf(uniform23(o.x)));
    const float r1 = sqrtf(-2.0f * logf(uniform23(o.z)));
    float s0, c0;
    sincospif(2.0f * uniform23(o.y), &s0, &c0);
    const float c1 = cospif(2.0f * uniform23(o.w));
    return make_float3(r0 * c0, r0 * s0, r1 * c1);
}

// The same three normals with the hardware sine, cosine and logarithm in
// place of sincospi / cospi / logf: the O-step noise of the FP32 dynamics
// kernels, where their errors (a few 1e-7 absolute) are far below the FP32
// rounding of the velocities.  cos(2 pi u) = -cos(2 pi (u - 1/2)) keeps the
// argument in [-pi, pi).  For the top one or two values of u the hardware
// logarithm of u (exactly ~ -6e-8) may come out positive: -2 ln u is clamped
// at 0, an error below 1e-3 in a normal on a set of probability ~2e-7.
__device__ __forceinline__ float3 normal3_fast(unsigned long long seed, uint32_t atom, uint32_t slot,
                                               uint32_t step, uint32_t purpose) {
    const uint4 o = philox4x32_10(make_uint4(atom, slot, step, purpose), seed_key(seed));
    const float r0 = sqrtf(fmaxf(-2.0f * __logf(uniform23(o.x)), 0.0f));
    const float r1 = sqrtf(fmaxf(-2.0f * __logf(uniform23(o.z)), 0.0f));
    const float two_pi = 6.2831853071795864769f;
    float s0, c0;
    __sincosf(two_pi * (uniform23(o.y) - 0.5f), &s0, &c0);
    const float c1 = __cosf(two_pi * (uniform23(o.w) - 0.5f));
    return make_float3(-r0 * c0, -r0 * s0, -r1 * c1);
}

// Taylor coefficients 1/n!, n = 0..13, filled on the host (correctly rounded
// binary64 divisions of exact factorials) and passed as a kernel argument.
struct ExpCoef {
    double c[14];
};

// e^x by Cody & Waite (1980) reduction x = k ln2 + r and the degree-13 Taylor
// polynomial of e^r in Horner form, every step an explicitly rounded binary64
// operation so that the result is the same on every IEEE machine.
__device__ __forceinline__ double exp_det(double x, const ExpCoef& cf) {
    if (x < -708.0) return 0.0;
    if (x > 709.0) return __longlong_as_double(0x7ff0000000000000LL);
    const double inv_ln2 = 0x1.71547652b82fep+0;
    const double ln2_hi = 0x1.62e42fee00000p-1;
    const double ln2_lo = 0x1.a39ef35793c76p-33;
    const double kf = rint(__dmul_rn(x, inv_ln2));
    double r = __fma_rn(-kf, ln2_hi, x);
    r = __fma_rn(-kf, ln2_lo, r);
    double p = cf.c[13];
#pragma unroll
    for (int n = 12; n >= 0; --n) p = __fma_rn(p, r, cf.c[n]);
    const long long k = (long long)kf;
    return __dmul_rn(p, __longlong_as_double((k + 1023LL) << 52));
}

}  // namespace pamd
