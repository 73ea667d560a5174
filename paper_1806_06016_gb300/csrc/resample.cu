// resample.cu -- population set-up, resampling, gather and observables.
//
// PAMD scheme, step 1 (init), step 2 (resampling with relative Boltzmann
// weights, velocity rescaling) and step 4 (population averages with
// family-binned errors).  Everything here is O(R) work between the
// propagate launches; the gather is the one HBM-bound kernel.
#include <math.h>

#include "pamd_device.cuh"
#include "pamd_internal.h"

namespace pamd {

constexpr int kScanBlock = 1024;  // elements per scan block (256 threads x 4)
constexpr int kScanThreads = 256;

// ------------------------------------------------------------------ helpers

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

// Inclusive scan of the 4 values held by each of the 256 threads (1024
// consecutive elements); returns the block total.
template <typename T>
__device__ __forceinline__ T block_scan4(T (&v)[4], T* sh /* [8] */) {
    v[1] += v[0];
    v[2] += v[1];
    v[3] += v[2];
    const T tsum = v[3];
    const T incl = warp_incl_scan(tsum);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 31) sh[w] = incl;
    __syncthreads();
    T wpre = 0, total = 0;
#pragma unroll
    for (int i = 0; i < kScanThreads / 32; ++i) {
        if (i < w) wpre += sh[i];
        total += sh[i];
    }
    const T pre = wpre + incl - tsum;
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] += pre;
    __syncthreads();
    return total;
}

__device__ __forceinline__ double block_max_d(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double m = -INFINITY;
    for (int i = 0; i < nw; ++i) m = fmax(m, sh[i]);
    __syncthreads();
    return m;
}

// Sum in a fixed tree order (deterministic for a given launch shape).
__device__ __forceinline__ double block_sum_d(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < nw; ++i) s += sh[i];
    __syncthreads();
    return s;
}

// ------------------------------------------------------------------ init

// Step 1: x = recentred start geometry, v ~ Maxwell-Boltzmann(T0) from
// Philox(seed; atom, slot, 0, INIT | mol << 8), family = slot.
__global__ void init_kernel(float* state, double* E, int32_t* fam, const float* x0,
                            const float* masses, long long R, int N, int Np, float kT0,
                            unsigned long long seed, uint32_t purpose) {
    const long long total = R * (long long)Np;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long k = t / Np;
        const int i = (int)(t - k * Np);
        float* st = state + (size_t)k * 6 * Np;
        if (i < N) {
            const float3 z = normal3(seed, (uint32_t)i, (uint32_t)k, 0u, purpose);
            const float sdv = sqrtf(kT0 / masses[i]);
            st[i] = x0[i];
            st[Np + i] = x0[Np + i];
            st[2 * Np + i] = x0[2 * Np + i];
            st[3 * Np + i] = sdv * z.x;
            st[4 * Np + i] = sdv * z.y;
            st[5 * Np + i] = sdv * z.z;
        } else {
#pragma unroll
            for (int c = 0; c < 6; ++c) st[c * Np + i] = 0.0f;
        }
        if (i == 0) {
            fam[k] = (int32_t)k;
            E[k] = 0.0;
        }
    }
}

__global__ void reset_scalars_kernel(DevScalars* s) {
    s->m = 0.0;
    s->S = 0.0;
    s->lnQ = 0.0;
    s->sum_lnQ = 0.0;
    s->C_total = 0ull;
    s->max_copies = 1;
    s->status = 0;
    s->bad_replica = -1;
}

__global__ void set_counters_kernel(uint32_t* ctr, uint32_t step, uint32_t ridx) {
    ctr[0] = step;
    ctr[1] = ridx;
}

// Population size of a context with a variable population (device counter
// word 2, read by every kernel that loops over the population).
__global__ void set_live_kernel(uint32_t* ctr, uint32_t live) { ctr[2] = live; }

// Live population size: *live when the population size varies, else R.
__device__ __forceinline__ long long live_size(const uint32_t* live, long long R) {
    return live ? (long long)*live : R;
}

// ------------------------------------------------------------------ weights

// a_j = -(beta_next - beta_prev) E_j ; block maxima.
__global__ void amax_kernel(const double* E, long long R, double dbeta, double* blk_max,
                            const uint32_t* live) {
    __shared__ double sh[32];
    R = live_size(live, R);
    const long long base = (long long)blockIdx.x * kScanBlock;
    double m = -INFINITY;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const long long j = base + threadIdx.x * 4 + q;
        if (j < R && isfinite(E[j])) m = fmax(m, __dmul_rn(-dbeta, E[j]));
    }
    m = block_max_d(m, sh);
    if (threadIdx.x == 0) blk_max[blockIdx.x] = m;
}

__global__ void max_top_kernel(const double* blk_max, int nblk, DevScalars* s) {
    __shared__ double sh[32];
    double m = -INFINITY;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) m = fmax(m, blk_max[b]);
    m = block_max_d(m, sh);
    if (threadIdx.x == 0) s->m = m;
}

// W_j = floor(2^s exp_det(a_j - m)); block sums of W (exact) and of the
// exponentials (for Q).
__global__ void weights_kernel(const double* E, long long R, double dbeta, double two_s,
                               DevScalars* s, ExpCoef cf, unsigned long long* W,
                               unsigned long long* blk_w, double* blk_e, const uint32_t* live) {
    __shared__ double sh[32];
    __shared__ unsigned long long shw[8];
    if (live) {  // 2^s with s = 63 - ceil(log2 R) of the live population
        R = (long long)*live;
        const int bits = (R > 1) ? 64 - __clzll((unsigned long long)(R - 1)) : 0;
        two_s = ldexp(1.0, 63 - bits);
    }
    const long long base = (long long)blockIdx.x * kScanBlock;
    const double m = s->m;
    unsigned long long w[4];
    double es = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const long long j = base + threadIdx.x * 4 + q;
        w[q] = 0ull;
        if (j < R) {
            const double Ej = E[j];
            double e = 0.0;
            if (isfinite(Ej)) {
                const double a = __dmul_rn(-dbeta, Ej);
                e = exp_det(__dsub_rn(a, m), cf);
                w[q] = __double2ull_rz(__dmul_rn(two_s, e));
            } else if (atomicCAS(&s->status, 0, PAMD_ENONFINITE) == 0) {
                s->bad_replica = (int)j;  // a non-finite energy gets weight 0
            }
            W[j] = w[q];
            es += e;
        }
    }
    const double bs = block_sum_d(es, sh);
    const unsigned long long tot = block_scan4(w, shw);
    if (threadIdx.x == 0) {
        blk_w[blockIdx.x] = tot;
        blk_e[blockIdx.x] = bs;
    }
}

// Exclusive scan of the block sums of W (in place), C_total, ln Q.
__global__ void weights_top_kernel(unsigned long long* blk_w, const double* blk_e, int nblk,
                                   long long R, DevScalars* s, const uint32_t* live) {
    R = live_size(live, R);
    __shared__ unsigned long long shw[8];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0ull;
    __syncthreads();
    for (int b0 = 0; b0 < nblk; b0 += kScanBlock) {
        unsigned long long v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int b = b0 + threadIdx.x * 4 + q;
            v[q] = (b < nblk) ? blk_w[b] : 0ull;
        }
        unsigned long long orig[4] = {v[0], v[1], v[2], v[3]};
        const unsigned long long tot = block_scan4(v, shw);
        const unsigned long long c = carry;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int b = b0 + threadIdx.x * 4 + q;
            if (b < nblk) blk_w[b] = c + v[q] - orig[q];
        }
        __syncthreads();
        if (threadIdx.x == 0) carry = c + tot;
        __syncthreads();
    }
    // S = sum of the block sums in a fixed order: each thread a contiguous
    // chunk, then a fixed shuffle tree per warp, then the warps in order
    __shared__ double wsum[32];
    double part = 0.0;
    {
        const int per = (nblk + blockDim.x - 1) / blockDim.x;
        const int lo = threadIdx.x * per, hi = min(lo + per, nblk);
        for (int b = lo; b < hi; ++b) part += blk_e[b];
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double S = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) S += wsum[w];
        s->S = S;
        s->C_total = carry;
        const double lnq = s->m + (log(S) - log((double)R));
        s->lnQ = lnq;
        s->sum_lnQ += lnq;
    }
}

// C_j = block offset + inclusive scan of W inside the block.
__global__ void scan_local_u64_kernel(unsigned long long* W, long long R,
                                      const unsigned long long* blk_off, unsigned long long* C,
                                      const uint32_t* live) {
    __shared__ unsigned long long shw[8];
    R = live_size(live, R);
    const long long base = (long long)blockIdx.x * kScanBlock;
    unsigned long long v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const long long j = base + threadIdx.x * 4 + q;
        v[q] = (j < R) ? W[j] : 0ull;
    }
    block_scan4(v, shw);
    const unsigned long long off = blk_off[blockIdx.x];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const long long j = base + threadIdx.x * 4 + q;
        if (j < R) C[j] = off + v[q];
    }
}

// ------------------------------------------------------------------ counts

// Draw k: u_k from Philox(seed; k, resampling index, 0, RESAMPLE | mol << 8),
// target t = floor(u_k C_total / 2^64), ancestor = first j with C_j > t.
__global__ void counts_kernel(const unsigned long long* C, long long R, const DevScalars* s,
                              unsigned long long seed, const uint32_t* dev_counters,
                              uint32_t ridx_off, uint32_t purpose, int do_resample,
                              int32_t* cnt, const uint32_t* live) {
    R = live_size(live, R);
    const uint32_t ridx = (dev_counters ? dev_counters[1] : 0u) + ridx_off;
    const unsigned long long total = s->C_total;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < R;
         k += (long long)gridDim.x * blockDim.x) {
        if (!do_resample) {
            cnt[k] = 1;
            continue;
        }
        unsigned long long t;
        if (do_resample == 2) {
            // systematic: t_k = floor((k C + V) / R), V = floor(u_0 C / 2^64), by
            // long division in 32-bit digits (the numerator is below 2^84 and
            // the quotient below C)
            const uint4 o = philox4x32_10(make_uint4(0u, ridx, 0u, purpose), seed_key(seed));
            const unsigned long long u0 = (unsigned long long)o.x | ((unsigned long long)o.y << 32);
            const unsigned long long V = __umul64hi(u0, total);
            const unsigned long long plo = (unsigned long long)k * total;  // low 64 bits of k C
            unsigned long long phi = __umul64hi((unsigned long long)k, total);
            const unsigned long long lo64 = plo + V;
            phi += (lo64 < plo) ? 1ull : 0ull;
            const unsigned long long r64 = (unsigned long long)R;
            unsigned long long rem = phi % r64;  // phi < R: the quotient's high word is zero
            unsigned long long cur = (rem << 32) | (lo64 >> 32);
            const unsigned long long q1 = cur / r64;
            rem = cur % r64;
            cur = (rem << 32) | (lo64 & 0xffffffffull);
            const unsigned long long q0 = cur / r64;
            t = (q1 << 32) | q0;
        } else {
            const uint4 o = philox4x32_10(make_uint4((uint32_t)k, ridx, 0u, purpose), seed_key(seed));
            const unsigned long long u = (unsigned long long)o.x | ((unsigned long long)o.y << 32);
            t = __umul64hi(u, total);
        }
        long long lo = 0, hi = R;
        while (lo < hi) {
            const long long mid = lo + ((hi - lo) >> 1);
            if (C[mid] > t) hi = mid;
            else lo = mid + 1;
        }
        // t < C_total whenever C_total > 0, so lo < R; the clamp only guards
        // a population whose weights are all zero (all energies non-finite)
        atomicAdd(&cnt[lo < R ? lo : R - 1], 1);
    }
}

// ------------------------------------------------------------------ copy numbers
// of the rules that let the population size vary around a target R_t

// q = floor(a b / c), r = a b - q c exactly, for a < 2^32, b <= c, c >= 1:
// an FP64 estimate corrected in 128-bit integer arithmetic.
__device__ __forceinline__ void muldiv_exact(unsigned long long a, unsigned long long b,
                                             unsigned long long c, unsigned long long& q,
                                             unsigned long long& r) {
    const unsigned long long plo = a * b, phi = __umul64hi(a, b);
    unsigned long long qq = (unsigned long long)__ddiv_rn(
        __dmul_rn(__ull2double_rn(a), __ull2double_rn(b)), __ull2double_rn(c));
    for (int it = 0; it < 8; ++it) {
        const unsigned long long tlo = qq * c, thi = __umul64hi(qq, c);
        if (thi > phi || (thi == phi && tlo > plo)) {  // qq c > a b
            --qq;
            continue;
        }
        const unsigned long long rlo = plo - tlo;
        const unsigned long long rhi = phi - thi - (plo < tlo ? 1ull : 0ull);
        if (rhi == 0ull && rlo < c) {
            q = qq;
            r = rlo;
            return;
        }
        ++qq;
    }
    q = qq;  // not reached: the estimate is within one of the quotient
    r = 0ull;
}

// Smallest n with F(n) >= u for the Poisson CDF F of mean lam, summed as
// p_0 = e^-lam, p_n = (p_{n-1} lam) / n (every operation rounded to FP64 as
// written); at most floor(lam + 20 sqrt(lam)) + 50.
__device__ __forceinline__ long long poisson_inverse(double lam, double u, const ExpCoef& cf) {
    const long long n_max = (long long)floor(__dadd_rn(lam, __dmul_rn(20.0, __dsqrt_rn(lam)))) + 50;
    double p = exp_det(-lam, cf);
    double F = p;
    long long n = 0;
    while (u > F && n < n_max) {
        ++n;
        p = __ddiv_rn(__dmul_rn(p, lam), (double)n);
        F = __dadd_rn(F, p);
    }
    return n;
}

// Copy numbers of ancestor j with E[n_j] = tau_j = R_t W_j / C (C = sum of
// the integer weights W of the live population): rule 3 nearest integer
// (floor(tau_j) plus a Bernoulli draw of the fractional part), rule 4
// Poisson (CDF inversion, in chunks of at most 500 of the mean).
__global__ void varsize_counts_kernel(const unsigned long long* W, long long R, const DevScalars* s,
                                      long long R_target, unsigned long long seed,
                                      const uint32_t* dev_counters, uint32_t ridx_off,
                                      uint32_t purpose, int rule, ExpCoef cf, int32_t* cnt,
                                      const uint32_t* live) {
    R = live_size(live, R);
    const uint32_t ridx = (dev_counters ? dev_counters[1] : 0u) + ridx_off;
    const unsigned long long C = s->C_total;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < R;
         j += (long long)gridDim.x * blockDim.x) {
        long long n = 0;
        if (C > 0ull && rule == 3) {
            unsigned long long q, r;
            muldiv_exact((unsigned long long)R_target, W[j], C, q, r);
            const uint4 o = philox4x32_10(make_uint4((uint32_t)j, ridx, 0u, purpose), seed_key(seed));
            const unsigned long long u = (unsigned long long)o.x | ((unsigned long long)o.y << 32);
            n = (long long)q + ((__umul64hi(u, C) < r) ? 1 : 0);
        } else if (C > 0ull) {
            const double lam = __ddiv_rn(__dmul_rn((double)R_target, __ull2double_rn(W[j])),
                                         __ull2double_rn(C));
            int m = (int)ceil(__ddiv_rn(lam, 500.0));
            m = m < 1 ? 1 : m;
            const double chunk = __ddiv_rn(lam, (double)m);
            for (int c = 0; c < m; ++c) {
                const uint4 o = philox4x32_10(make_uint4((uint32_t)j, ridx, (uint32_t)c, purpose),
                                              seed_key(seed));
                const unsigned long long u64 = (unsigned long long)o.x | ((unsigned long long)o.y << 32);
                const double u = __dmul_rn(__dadd_rn(__ull2double_rn(u64 >> 11), 0.5), 0x1p-53);
                n += poisson_inverse(chunk, u, cf);
            }
        }
        cnt[j] = (int32_t)n;
    }
}

// After the gather: the new population size becomes the live size (at most
// the capacity R); an empty or overflowing population is reported.
__global__ void commit_size_kernel(DevScalars* s, uint32_t* ctr, long long R) {
    const long long n = s->R_new;
    if ((n == 0 || n > R) && atomicCAS(&s->status, 0, PAMD_EPOPSIZE) == 0) s->bad_replica = -1;
    ctr[2] = (uint32_t)(n < R ? n : R);
}

__global__ void cnt_block_kernel(const int32_t* cnt, long long R, int32_t* blk_sum,
                                 int32_t* blk_max, const uint32_t* live) {
    R = live_size(live, R);
    __shared__ int32_t shs[8];
    __shared__ int32_t shm[8];
    const long long base = (long long)blockIdx.x * kScanBlock;
    int32_t v[4], mx = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const long long j = base + threadIdx.x * 4 + q;
        v[q] = (j < R) ? cnt[j] : 0;
        mx = max(mx, v[q]);
    }
    const int32_t tot = block_scan4(v, shs);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t m = 0;
        for (int i = 0; i < kScanThreads / 32; ++i) m = max(m, shm[i]);
        blk_sum[blockIdx.x] = tot;
        blk_max[blockIdx.x] = m;
    }
}

__global__ void cnt_top_kernel(int32_t* blk_sum, const int32_t* blk_max, int nblk, DevScalars* s) {
    __shared__ int32_t shs[8];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nblk; b0 += kScanBlock) {
        int32_t v[4], orig[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int b = b0 + threadIdx.x * 4 + q;
            v[q] = orig[q] = (b < nblk) ? blk_sum[b] : 0;
        }
        const int32_t tot = block_scan4(v, shs);
        const int32_t c = carry;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int b = b0 + threadIdx.x * 4 + q;
            if (b < nblk) blk_sum[b] = c + v[q] - orig[q];
        }
        __syncthreads();
        if (threadIdx.x == 0) carry = c + tot;
        __syncthreads();
    }
    // largest count: an integer max, the same in any order
    __shared__ int32_t wmax[32];
    int32_t mloc = 0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) mloc = max(mloc, blk_max[b]);
    for (int o = 16; o > 0; o >>= 1) mloc = max(mloc, __shfl_down_sync(0xffffffffu, mloc, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mloc;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t m = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, wmax[w]);
        s->max_copies = m;
        s->R_new = carry;  // size of the new population (sum of the copy counts)
    }
}

__global__ void cnt_local_kernel(const int32_t* cnt, long long R, const int32_t* blk_off,
                                 int32_t* incl, const uint32_t* live) {
    __shared__ int32_t shs[8];
    R = live_size(live, R);
    const long long base = (long long)blockIdx.x * kScanBlock;
    int32_t v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const long long j = base + threadIdx.x * 4 + q;
        v[q] = (j < R) ? cnt[j] : 0;
    }
    block_scan4(v, shs);
    const int32_t off = blk_off[blockIdx.x];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const long long j = base + threadIdx.x * 4 + q;
        if (j < R) incl[j] = off + v[q];
    }
}

// ------------------------------------------------------------------ gather

// Ancestor of every new slot: anc[k] = first j with incl_j > k (copies of j
// fill slots incl_{j-1} .. incl_j - 1).  One thread per slot.
// With a variable population (live != null) the ancestors are the live
// population and the new slots number min(R_new, R), R the capacity.
__global__ void ancestor_kernel(const int32_t* __restrict__ incl, long long R, int32_t* anc,
                                const uint32_t* live, const DevScalars* s) {
    long long n_new = R;
    if (live) {
        n_new = s->R_new < R ? s->R_new : R;
        R = (long long)*live;
    }
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n_new;
         k += (long long)gridDim.x * blockDim.x) {
        long long lo = 0, hi = R;
        while (lo < hi) {
            const long long mid = lo + ((hi - lo) >> 1);
            if (incl[mid] > k) hi = mid;
            else lo = mid + 1;
        }
        anc[k] = (int32_t)(lo < R ? lo : R - 1);
    }
}

// One warp per new slot k copies the ancestor's state (6 Np floats, Np % 4 ==
// 0) as P float4s per lane: positions shifted to the centre of mass,
// velocities scaled by vscale, and the new replica's kinetic energy and
// radius of gyration recomputed from the moved state (FP32 sums: GB300's FP64
// rate is a small fraction of its FP32 rate, and every propagate launch
// recomputes these values in FP64).
template <int P>
__global__ void __launch_bounds__(256) gather_kernel(
    const float* __restrict__ st_in, float* __restrict__ st_out, const double* E_in,
    double* E_out, const int32_t* fam_in, int32_t* fam_out, double* ke_out, double* rg_out,
    const int32_t* __restrict__ anc, const float* __restrict__ masses, long long R, int N, int Np,
    float vscale, float inv_mtot, const uint32_t* live, const DevScalars* sc) {
    const int lane = threadIdx.x & 31;
    if (live) R = sc->R_new < R ? sc->R_new : R;  // new slots of a variable population
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int q4 = Np / 4;          // float4s per component
    const int nq = 6 * q4;          // float4s per replica
    const float4* m4 = reinterpret_cast<const float4*>(masses);
    for (long long k = warp; k < R; k += nwarps) {
        const long long j = anc[k];
        const float4* src = reinterpret_cast<const float4*>(st_in + (size_t)j * 6 * Np);
        float4* dst = reinterpret_cast<float4*>(st_out + (size_t)k * 6 * Np);
        float4 v[P];
#pragma unroll
        for (int r = 0; r < P; ++r) {
            const int q = lane + 32 * r;
            if (q < nq) v[r] = __ldcs(src + q);  // read once: streaming load
        }
        float sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
        for (int r = 0; r < P; ++r) {
            const int q = lane + 32 * r;
            if (q < nq) {
                const int comp = q / q4;
                if (comp < 3) {
                    const float4 m = m4[q - comp * q4];
                    const float s = m.x * v[r].x + m.y * v[r].y + m.z * v[r].z + m.w * v[r].w;
                    sx += comp == 0 ? s : 0.f;
                    sy += comp == 1 ? s : 0.f;
                    sz += comp == 2 ? s : 0.f;
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
            sz += __shfl_xor_sync(0xffffffffu, sz, o);
        }
        const float cx = sx * inv_mtot, cy = sy * inv_mtot, cz = sz * inv_mtot;
        float mv2 = 0.f, ux = 0.f, uy = 0.f, uz = 0.f, u2 = 0.f;
#pragma unroll
        for (int r = 0; r < P; ++r) {
            const int q = lane + 32 * r;
            if (q < nq) {
                const int comp = q / q4;
                const int i0 = (q - comp * q4) * 4;
                float4 w = v[r];
                const float4 m = m4[q - comp * q4];  // 0 for padding atoms
                // padding atoms (i >= N) are kept out of the sums
                const float4 real = make_float4(i0 < N ? 1.f : 0.f, i0 + 1 < N ? 1.f : 0.f,
                                                i0 + 2 < N ? 1.f : 0.f, i0 + 3 < N ? 1.f : 0.f);
                if (comp < 3) {
                    const float c = (comp == 0) ? cx : (comp == 1) ? cy : cz;
                    w.x -= c; w.y -= c; w.z -= c; w.w -= c;
                    const float s1 = real.x * w.x + real.y * w.y + real.z * w.z + real.w * w.w;
                    u2 += real.x * w.x * w.x + real.y * w.y * w.y + real.z * w.z * w.z + real.w * w.w * w.w;
                    ux += comp == 0 ? s1 : 0.f;
                    uy += comp == 1 ? s1 : 0.f;
                    uz += comp == 2 ? s1 : 0.f;
                } else {
                    w.x *= vscale; w.y *= vscale; w.z *= vscale; w.w *= vscale;
                    mv2 += m.x * w.x * w.x + m.y * w.y * w.y + m.z * w.z * w.z + m.w * w.w * w.w;
                }
                __stcs(dst + q, w);  // written once: streaming store
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mv2 += __shfl_xor_sync(0xffffffffu, mv2, o);
            ux += __shfl_xor_sync(0xffffffffu, ux, o);
            uy += __shfl_xor_sync(0xffffffffu, uy, o);
            uz += __shfl_xor_sync(0xffffffffu, uz, o);
            u2 += __shfl_xor_sync(0xffffffffu, u2, o);
        }
        if (lane == 0) {
            E_out[k] = E_in[j];
            fam_out[k] = fam_in[j];
            ke_out[k] = 0.5 * (double)mv2;
            const float mx = ux / N, my = uy / N, mz = uz / N;
            rg_out[k] = (double)sqrtf(fmaxf(u2 / N - (mx * mx + my * my + mz * mz), 0.f));
        }
    }
}

// ------------------------------------------------------------------ observables

// Family ids lie in 0 .. R-1 (R the slots of the population buffers); the
// live replicas are the first live_size(live, R).
__global__ void mark_kernel(const int32_t* fam, long long R, unsigned char* flags,
                            const uint32_t* live) {
    const long long n = live_size(live, R);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int32_t f = fam[k];
        if (f >= 0 && f < R) flags[f] = 1;
    }
}

constexpr int kObsVals = 5;  // count, E, E_kin, R_g, R_g^2
constexpr int kObsStride = kNumBins * kObsVals + 1;

// Partial sums per family bin over 1024 replicas, in replica order per bin.
// Per-bin partial sums of one 1024-replica chunk.  Each bin's sums are
// accumulated by one thread over the chunk's replicas of that bin in
// increasing index order.  The replicas are first ordered by bin with a
// stable counting sort (ranks within 32-replica pieces from
// __match_any_sync, prefix counts over the pieces), so that the 64 bin
// threads run side by side over their own segments instead of each scanning
// the whole chunk.
__global__ void obs_partial_kernel(const int32_t* fam, const double* E, const double* ke,
                                   const double* rg, const unsigned char* flags, long long R,
                                   double* part, const uint32_t* live) {
    constexpr int kPieces = kScanBlock / 32;
    constexpr int kPerWarp = kPieces / (kScanThreads / 32);
    static_assert(kPieces % (kScanThreads / 32) == 0, "pieces per warp");
    const long long n = live_size(live, R);  // replicas; family flags span R
    __shared__ int32_t sf[kScanBlock];
    __shared__ double se[kScanBlock], sk[kScanBlock], sr[kScanBlock];
    __shared__ int32_t famcount[kScanThreads / 32];
    __shared__ int32_t pcount[kPieces][kNumBins];  // per piece and bin: count, then prefix
    __shared__ int32_t bstart[kNumBins + 1];
    __shared__ int16_t order[kScanBlock];          // chunk entries sorted by bin (stable)
    const long long base = (long long)blockIdx.x * kScanBlock;
    int fc = 0;
    for (int t = threadIdx.x; t < kScanBlock; t += blockDim.x) {
        const long long k = base + t;
        if (k < n) {
            sf[t] = fam[k] & (kNumBins - 1);
            se[t] = E[k];
            sk[t] = ke[k];
            sr[t] = rg[k];
        } else {
            sf[t] = -1;
        }
        if (k < R) fc += flags[k];
    }
    for (int i = threadIdx.x; i < kPieces * kNumBins; i += blockDim.x) (&pcount[0][0])[i] = 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fc += __shfl_xor_sync(0xffffffffu, fc, o);
    if ((threadIdx.x & 31) == 0) famcount[threadIdx.x >> 5] = fc;
    __syncthreads();
    // ranks within each piece, and the pieces' counts per bin
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int rank[kPerWarp];
#pragma unroll
    for (int q = 0; q < kPerWarp; ++q) {
        const int c = w + q * (kScanThreads / 32);
        const int bin = sf[32 * c + lane];
        const unsigned peers = __match_any_sync(0xffffffffu, bin);
        rank[q] = __popc(peers & ((1u << lane) - 1u));
        if (bin >= 0 && rank[q] == 0) pcount[c][bin] = __popc(peers);
    }
    __syncthreads();
    if (threadIdx.x < kNumBins) {  // prefix over the pieces, per bin
        int s = 0;
        for (int c = 0; c < kPieces; ++c) {
            const int x = pcount[c][threadIdx.x];
            pcount[c][threadIdx.x] = s;
            s += x;
        }
        bstart[threadIdx.x + 1] = s;  // the bin's size, turned into starts below
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        bstart[0] = 0;
        for (int b = 0; b < kNumBins; ++b) {
            s += bstart[b + 1];
            bstart[b + 1] = s;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kPerWarp; ++q) {
        const int c = w + q * (kScanThreads / 32);
        const int t = 32 * c + lane;
        const int bin = sf[t];
        if (bin >= 0) order[bstart[bin] + pcount[c][bin] + rank[q]] = (int16_t)t;
    }
    __syncthreads();
    double* out = part + (size_t)blockIdx.x * kObsStride;
    if (threadIdx.x < kNumBins) {
        const int b = threadIdx.x;
        double c = 0, e = 0, k2 = 0, r = 0, r2 = 0;
        for (int i = bstart[b]; i < bstart[b + 1]; ++i) {
            const int t = order[i];
            c += 1.0;
            e += se[t];
            k2 += sk[t];
            r += sr[t];
            r2 += sr[t] * sr[t];
        }
        out[b * kObsVals + 0] = c;
        out[b * kObsVals + 1] = e;
        out[b * kObsVals + 2] = k2;
        out[b * kObsVals + 3] = r;
        out[b * kObsVals + 4] = r2;
    }
    if (threadIdx.x == 0) {
        int s = 0;
        for (int i = 0; i < kScanThreads / 32; ++i) s += famcount[i];
        out[kNumBins * kObsVals] = (double)s;
    }
}

// Jackknife standard error over the family bins from the leave-one-bin-out
// means jk[b] (computed in parallel by the caller), bins that are empty or
// hold the whole population left out; the sums run over the bins in order.
__device__ double jackknife_se(const double* cnt, const double* jk, double R) {
    int nb = 0;
    double jm = 0.0;
    for (int b = 0; b < kNumBins; ++b) {
        if (cnt[b] == 0.0 || cnt[b] == R) continue;
        jm += jk[b];
        ++nb;
    }
    if (nb < 2) return 0.0;
    jm /= nb;
    double ss = 0.0;
    for (int b = 0; b < kNumBins; ++b) {
        if (cnt[b] == 0.0 || cnt[b] == R) continue;
        ss += (jk[b] - jm) * (jk[b] - jm);
    }
    return sqrt((double)(nb - 1) / nb * ss);
}

__global__ void obs_final_kernel(const double* part, int nblk, long long R, int N, double T,
                                 const DevScalars* s, pamd_obs* dst, const uint32_t* live) {
    R = live_size(live, R);
    __shared__ double bins[kObsVals][kNumBins];
    __shared__ double jk[kObsVals][kNumBins];
    __shared__ double tot[kObsVals];
    __shared__ double nfam;
    if (threadIdx.x < kNumBins) {
        const int b = threadIdx.x;
        double acc[kObsVals] = {0, 0, 0, 0, 0};
        for (int blk = 0; blk < nblk; ++blk)
            for (int v = 0; v < kObsVals; ++v) acc[v] += part[(size_t)blk * kObsStride + b * kObsVals + v];
        for (int v = 0; v < kObsVals; ++v) bins[v][b] = acc[v];
    }
    if (threadIdx.x == kNumBins) {
        double f = 0;
        for (int blk = 0; blk < nblk; ++blk) f += part[(size_t)blk * kObsStride + kNumBins * kObsVals];
        nfam = f;
    }
    __syncthreads();
    if (threadIdx.x >= 1 && threadIdx.x < kObsVals) {  // totals over the bins, in bin order
        const int v = threadIdx.x;
        double t = 0;
        for (int b = 0; b < kNumBins; ++b) t += bins[v][b];
        tot[v] = t;
    }
    __syncthreads();
    const double Rd = (double)R;
    if (threadIdx.x < kNumBins) {  // leave-one-bin-out means
        const int b = threadIdx.x;
        for (int v = 1; v < kObsVals; ++v) jk[v][b] = (tot[v] - bins[v][b]) / (Rd - bins[0][b]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        pamd_obs o;
        o.T = T;
        o.lnQ = s->lnQ;
        o.sum_lnQ = s->sum_lnQ;
        o.e_pot = tot[1] / Rd;
        o.e_pot_se = jackknife_se(bins[0], jk[1], Rd);
        o.e_kin = tot[2] / Rd;
        o.e_kin_se = jackknife_se(bins[0], jk[2], Rd);
        o.t_meas = 2.0 * o.e_kin / (3.0 * N * kBoltzmann);
        o.rg = tot[3] / Rd;
        o.rg_se = jackknife_se(bins[0], jk[3], Rd);
        o.rg2 = tot[4] / Rd;
        o.rg2_se = jackknife_se(bins[0], jk[4], Rd);
        o.n_families = (int64_t)nfam;
        o.max_copies = s->max_copies;
        o.pad_ = s->status;
        o.R_live = R;
        *dst = o;
    }
}

// ------------------------------------------------------------------ host side

static int grid_for(long long n, int threads, int cap) {
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

cudaError_t launch_init(pamd_ctx* c, double T0) {
    if (c->precision == PAMD_PREC_FP64) {
        const cudaError_t e = launch_init_f64(c, T0);
        if (e != cudaSuccess) return e;
        reset_scalars_kernel<<<1, 1, 0, c->stream>>>(c->b.scal);
        c->launches += 1;
        return cudaGetLastError();
    }
    const long long total = c->R * c->Np;
    init_kernel<<<grid_for(total, 256, c->num_sms * 16), 256, 0, c->stream>>>(
        c->b.state, c->b.E, c->b.fam, c->b.x0, c->b.masses, c->R, c->N, c->Np,
        (float)(kBoltzmann * T0), c->seed, kPurposeInit | ((uint32_t)c->mol << 8));
    reset_scalars_kernel<<<1, 1, 0, c->stream>>>(c->b.scal);
    c->launches += 2;
    if (c->variable) {  // the population starts at its target size
        set_live_kernel<<<1, 1, 0, c->stream>>>(c->b.counters, (uint32_t)c->R_target);
        c->launches += 1;
    }
    return cudaGetLastError();
}

cudaError_t launch_set_counters(pamd_ctx* c, uint32_t step, uint32_t ridx) {
    set_counters_kernel<<<1, 1, 0, c->stream>>>(c->b.counters, step, ridx);
    c->launches += 1;
    return cudaGetLastError();
}

static ExpCoef exp_coefficients() {
    ExpCoef cf;
    double f = 1.0;
    for (int n = 0; n < 14; ++n) {
        if (n > 0) f *= (double)n;
        cf.c[n] = 1.0 / f;
    }
    return cf;
}

cudaError_t launch_resample(pamd_ctx* c, double T_prev, double T_next, int do_resample,
                            const uint32_t* dev_counters, uint32_t resample_offset) {
    // R: slots of the population buffers (the capacity of a variable
    // population, whose live size the kernels read from counter word 2)
    const long long R = c->R;
    const uint32_t* live = c->variable ? c->b.counters + 2 : nullptr;
    const int nblk = c->n_blk;
    cudaStream_t s = c->stream;
    const double dbeta = 1.0 / (kBoltzmann * T_next) - 1.0 / (kBoltzmann * T_prev);
    int bits = 0;
    while ((1LL << bits) < R) ++bits;
    const double two_s = ldexp(1.0, 63 - bits);
    static const ExpCoef cf = exp_coefficients();

    // energies of the current population (the ping-pong buffers alternate)
    const double* Ecur = c->cur_is_alt ? c->b.E_alt : c->b.E;
    amax_kernel<<<nblk, kScanThreads, 0, s>>>(Ecur, R, dbeta, c->b.blk_f64, live);
    max_top_kernel<<<1, 1024, 0, s>>>(c->b.blk_f64, nblk, c->b.scal);
    weights_kernel<<<nblk, kScanThreads, 0, s>>>(Ecur, R, dbeta, two_s, c->b.scal, cf, c->b.W,
                                                 c->b.blk_u64, c->b.blk_f64, live);
    weights_top_kernel<<<1, kScanThreads, 0, s>>>(c->b.blk_u64, c->b.blk_f64, nblk, R, c->b.scal, live);
    scan_local_u64_kernel<<<nblk, kScanThreads, 0, s>>>(c->b.W, R, c->b.blk_u64, c->b.C, live);
    cudaError_t e = cudaMemsetAsync(c->b.cnt, 0, sizeof(int32_t) * (size_t)R, s);
    if (e != cudaSuccess) return e;
    if (c->variable && do_resample) {
        varsize_counts_kernel<<<grid_for(R, 256, c->num_sms * 16), 256, 0, s>>>(
            c->b.W, R, c->b.scal, c->R_target, c->seed, dev_counters, resample_offset,
            kPurposeResample | ((uint32_t)c->mol << 8),
            c->resample_rule == PAMD_RESAMPLE_NEAREST ? 3 : 4, cf, c->b.cnt, live);
    } else {
        const int rule = !do_resample ? 0 : (c->resample_rule == PAMD_RESAMPLE_SYSTEMATIC ? 2 : 1);
        counts_kernel<<<grid_for(R, 256, c->num_sms * 16), 256, 0, s>>>(
            c->b.C, R, c->b.scal, c->seed, dev_counters, resample_offset,
            kPurposeResample | ((uint32_t)c->mol << 8), rule, c->b.cnt, live);
    }
    cnt_block_kernel<<<nblk, kScanThreads, 0, s>>>(c->b.cnt, R, c->b.blk_i32, c->b.blk_i32 + nblk, live);
    cnt_top_kernel<<<1, kScanThreads, 0, s>>>(c->b.blk_i32, c->b.blk_i32 + nblk, nblk, c->b.scal);
    cnt_local_kernel<<<nblk, kScanThreads, 0, s>>>(c->b.cnt, R, c->b.blk_i32, c->b.cnt_incl, live);
    double mt = 0.0;
    for (double m : c->host_mass) mt += m;
    const float* src = c->cur_is_alt ? c->b.state_alt : c->b.state;
    float* dst = c->cur_is_alt ? c->b.state : c->b.state_alt;
    const double* Ein = c->cur_is_alt ? c->b.E_alt : c->b.E;
    double* Eout = c->cur_is_alt ? c->b.E : c->b.E_alt;
    const int32_t* fin = c->cur_is_alt ? c->b.fam_alt : c->b.fam;
    int32_t* fout = c->cur_is_alt ? c->b.fam : c->b.fam_alt;
    if (c->precision == PAMD_PREC_FP64) {
        const cudaError_t e = launch_gather_f64(
            c, reinterpret_cast<const double*>(src), reinterpret_cast<double*>(dst), Ein, Eout, fin,
            fout, sqrt(T_next / T_prev));
        c->launches += 9;
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    // ancestors of the new slots (into the weight buffer, no longer needed)
    int32_t* anc = reinterpret_cast<int32_t*>(c->b.W);
    ancestor_kernel<<<grid_for(R, 256, c->num_sms * 16), 256, 0, s>>>(c->b.cnt_incl, R, anc, live,
                                                                       c->b.scal);
    const int gridg = grid_for(R * 32, 256, c->num_sms * 64);
    const float vs = (float)sqrt(T_next / T_prev), imt = (float)(1.0 / mt);
    switch ((6 * (c->Np / 4) + 31) / 32) {
#define PAMD_GATHER_CASE(P)                                                                     \
    case P:                                                                                     \
        gather_kernel<P><<<gridg, 256, 0, s>>>(src, dst, Ein, Eout, fin, fout, c->b.ke, c->b.rg, \
                                               anc, c->b.masses, R, c->N, c->Np, vs, imt, live, \
                                               c->b.scal);                                      \
        break;
        PAMD_GATHER_CASE(1) PAMD_GATHER_CASE(2) PAMD_GATHER_CASE(3) PAMD_GATHER_CASE(4)
        PAMD_GATHER_CASE(5) PAMD_GATHER_CASE(6) PAMD_GATHER_CASE(7) PAMD_GATHER_CASE(8)
        PAMD_GATHER_CASE(9) PAMD_GATHER_CASE(10) PAMD_GATHER_CASE(11) PAMD_GATHER_CASE(12)
#undef PAMD_GATHER_CASE
        default: return cudaErrorInvalidValue;
    }
    c->launches += 11;
    if (c->variable) {
        commit_size_kernel<<<1, 1, 0, s>>>(c->b.scal, c->b.counters, R);
        c->launches += 1;
    }
    return cudaGetLastError();
}

cudaError_t launch_observe(pamd_ctx* c, double T, pamd_obs* dst) {
    cudaStream_t s = c->stream;
    const long long R = c->R;
    const int32_t* fam = c->cur_is_alt ? c->b.fam_alt : c->b.fam;
    const double* E = c->cur_is_alt ? c->b.E_alt : c->b.E;
    cudaError_t e = cudaMemsetAsync(c->b.flags, 0, (size_t)R, s);
    if (e != cudaSuccess) return e;
    const uint32_t* live = c->variable ? c->b.counters + 2 : nullptr;
    mark_kernel<<<grid_for(R, 256, c->num_sms * 16), 256, 0, s>>>(fam, R, c->b.flags, live);
    obs_partial_kernel<<<c->n_blk, kScanThreads, 0, s>>>(fam, E, c->b.ke, c->b.rg, c->b.flags, R,
                                                        c->b.obs_part, live);
    obs_final_kernel<<<1, 128, 0, s>>>(c->b.obs_part, c->n_blk, R, c->N, T, c->b.scal, dst, live);
    c->launches += 3;
    return cudaGetLastError();
}

}  // namespace pamd
