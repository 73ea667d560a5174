// mlp_device.cuh -- block-level device helpers of the MLP energy surrogate:
// loading one configuration, its normalised inverse-distance features, and
// the force sum that maps de/dg back onto the atoms.
#pragma once

#include <cuda_bf16.h>

#include "mlp_internal.h"

namespace pamd {

constexpr int kXs = PAMD_MAX_ATOMS;  // stride of a coordinate row in shared memory

// index of pair (i, j), i < j, in row order
__device__ __forceinline__ int pair_id(int i, int j, int N) {
    return i * (2 * N - i - 1) / 2 + (j - i - 1);
}

__device__ __forceinline__ long long config_index(const ConfigView& cv, int m) {
    return cv.idx ? (long long)cv.idx[m] : (long long)m;
}

// xs[c * kXs + i] = coordinate c of atom i of configuration m (whole block)
__device__ __forceinline__ void load_config(const ConfigView& cv, int m, int N, float* xs) {
    const float* x = cv.x + config_index(cv, m) * cv.s_cfg;
    for (int t = threadIdx.x; t < 3 * N; t += blockDim.x) {
        int i, c;
        if (cv.s_coord == 1) {  // [N][3]: consecutive threads read consecutive floats
            i = t / 3;
            c = t - 3 * i;
        } else {
            c = t / N;
            i = t - c * N;
        }
        xs[c * kXs + i] = x[(long long)i * cv.s_atom + (long long)c * cv.s_coord];
    }
}

// a_p = (1 / r_ij - mu_p) / sd_p rounded to BF16, zero for the padding
// columns P <= p < Pp (whole block)
__device__ __forceinline__ void block_features(const float* xs, const ushort2* __restrict__ pairs,
                                               const float* __restrict__ mu,
                                               const float* __restrict__ inv_sd, int P, int Pp,
                                               __nv_bfloat16* a_row, __nv_bfloat16* aT, int ldt,
                                               int m) {
#pragma unroll 4
    for (int p = threadIdx.x; p < Pp; p += blockDim.x) {
        float v = 0.0f;
        if (p < P) {
            const ushort2 ij = pairs[p];
            const float dx = xs[ij.x] - xs[ij.y];
            const float dy = xs[kXs + ij.x] - xs[kXs + ij.y];
            const float dz = xs[2 * kXs + ij.x] - xs[2 * kXs + ij.y];
            const float g = rsqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
            v = (g - mu[p]) * inv_sd[p];
        }
        const __nv_bfloat16 b = __float2bfloat16(v);
        a_row[p] = b;
        if (aT) aT[(size_t)p * ldt + m] = b;
    }
}

// sum over j != k of gam_p(k,j) (x_k - x_j) / r_kj^3, i.e. minus the
// derivative of sum_p gam_p g_p with respect to x_k
__device__ __forceinline__ float3 atom_force(int k, const float* xs, const float* gam, int N) {
    const float xk = xs[k], yk = xs[kXs + k], zk = xs[2 * kXs + k];
    float fx = 0.0f, fy = 0.0f, fz = 0.0f;
    for (int j = 0; j < N; ++j) {
        if (j == k) continue;
        const int p = k < j ? pair_id(k, j, N) : pair_id(j, k, N);
        const float dx = xk - xs[j], dy = yk - xs[kXs + j], dz = zk - xs[2 * kXs + j];
        const float ir = rsqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
        const float c = gam[p] * ir * ir * ir;
        fx = fmaf(c, dx, fx);
        fy = fmaf(c, dy, fy);
        fz = fmaf(c, dz, fz);
    }
    return make_float3(fx, fy, fz);
}

// Molecules of up to kGammaMatrixMax atoms use a symmetric N x N shared-
// memory matrix (odd row stride: the atoms of a warp hit distinct banks)
// holding c_ij = gam_ij / r_ij^3, filled by one pass over the pairs (one
// rsqrt per pair), so that the force of atom k is the plain row sum
// F_k = sum_j c_kj (x_k - x_j).  Larger molecules keep gam per pair and use
// atom_force.  The diagonal is zero (set once per block, never written by
// the pair pass).
constexpr int kGammaMatrixMax = 128;

__host__ __device__ __forceinline__ bool gamma_matrix(int N) { return N <= kGammaMatrixMax; }
__host__ __device__ __forceinline__ int gamma_stride(int N) { return N | 1; }

// floats of shared memory the table of an N-atom molecule takes
__host__ __device__ __forceinline__ int gamma_floats(int N, int Pp) {
    return gamma_matrix(N) ? N * gamma_stride(N) : Pp;
}

// zero diagonal of the matrix (whole block; once per block)
__device__ __forceinline__ void init_gamma(int N, float* gam) {
    if (gamma_matrix(N))
        for (int k = threadIdx.x; k < N; k += blockDim.x) gam[k * gamma_stride(N) + k] = 0.0f;
}

// fill the table from de/da of one configuration (whole block)
__device__ __forceinline__ void load_gamma(const float* xs, const __nv_bfloat16* __restrict__ ga_row,
                                           const float* __restrict__ inv_sd,
                                           const ushort2* __restrict__ pairs, int P, int N, float* gam) {
    if (gamma_matrix(N)) {
        const int S = gamma_stride(N);
#pragma unroll 4
        for (int p = threadIdx.x; p < P; p += blockDim.x) {
            const ushort2 ij = pairs[p];
            const float dx = xs[ij.x] - xs[ij.y];
            const float dy = xs[kXs + ij.x] - xs[kXs + ij.y];
            const float dz = xs[2 * kXs + ij.x] - xs[2 * kXs + ij.y];
            const float ir = rsqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
            const float c = __bfloat162float(ga_row[p]) * inv_sd[p] * ir * ir * ir;
            gam[ij.x * S + ij.y] = c;
            gam[ij.y * S + ij.x] = c;
        }
    } else {
        for (int p = threadIdx.x; p < P; p += blockDim.x) gam[p] = __bfloat162float(ga_row[p]) * inv_sd[p];
    }
}

// sum over j != k of gam_kj (x_k - x_j) / r_kj^3 with the table of load_gamma
__device__ __forceinline__ float3 atom_force_any(int k, const float* xs, const float* gam, int N) {
    if (!gamma_matrix(N)) return atom_force(k, xs, gam, N);
    const float xk = xs[k], yk = xs[kXs + k], zk = xs[2 * kXs + k];
    const float* row = gam + k * gamma_stride(N);
    float fx = 0.0f, fy = 0.0f, fz = 0.0f;
#pragma unroll 4
    for (int j = 0; j < N; ++j) {
        const float c = row[j];
        fx = fmaf(c, xk - xs[j], fx);
        fy = fmaf(c, yk - xs[kXs + j], fy);
        fz = fmaf(c, zk - xs[2 * kXs + j], fz);
    }
    return make_float3(fx, fy, fz);
}

// ------------------------------------------------ pair passes of the MD step kernel
// Consecutive threads take consecutive row-order pairs, so that the lanes of
// a warp read consecutive atoms (no shared-memory bank conflicts) and
// consecutive table entries.  The pair table (i, j) and the per-pair tables
// may sit in shared or global memory.  Positions sit in shared memory as
// float4 (x, y, z, 0).  The arithmetic of every pair is that of
// block_features / load_gamma / atom_force_any, bit for bit.

__host__ __device__ __forceinline__ size_t step_pos_bytes(int N) { return 16 * (size_t)(N + 1); }

__device__ __forceinline__ float inv_dist4(const float4 a, const float4 b) {
    const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
    return rsqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
}

// positions of one replica from the population layout [6][Np] (whole block)
__device__ __forceinline__ void load_pos4(const float* st, int N, int Np, float4* xs4) {
    for (int i = threadIdx.x; i < N; i += blockDim.x)
        xs4[i] = make_float4(st[i], st[Np + i], st[2 * Np + i], 0.0f);
}

// features of the configuration in xs4 (whole block)
__device__ __forceinline__ void pass_features(const float4* xs4, const ushort2* pij, int P, int Pp,
                                              const float* mu, const float* inv_sd, __nv_bfloat16* a_row) {
#pragma unroll 4
    for (int p = threadIdx.x; p < Pp; p += blockDim.x) {
        float v = 0.0f;
        if (p < P) {
            const ushort2 ij = pij[p];
            v = (inv_dist4(xs4[ij.x], xs4[ij.y]) - mu[p]) * inv_sd[p];
        }
        a_row[p] = __float2bfloat16(v);
    }
}

// the table of load_gamma from de/da of the configuration in xs4 (whole block)
__device__ __forceinline__ void pass_gamma(const float4* xs4, const ushort2* pij, int P, int N,
                                           const __nv_bfloat16* ga_row, const float* inv_sd, float* gam) {
    if (!gamma_matrix(N)) {
        for (int p = threadIdx.x; p < P; p += blockDim.x) gam[p] = __bfloat162float(ga_row[p]) * inv_sd[p];
        return;
    }
    const int S = gamma_stride(N);
#pragma unroll 4
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        const ushort2 ij = pij[p];
        const float ir = inv_dist4(xs4[ij.x], xs4[ij.y]);
        const float c = __bfloat162float(ga_row[p]) * inv_sd[p] * ir * ir * ir;
        gam[ij.x * S + ij.y] = c;
        gam[ij.y * S + ij.x] = c;
    }
}

// sum over j != k of gam_kj (x_k - x_j) / r_kj^3 (atom_force_any on xs4)
__device__ __forceinline__ float3 atom_force4(int k, const float4* xs4, const float* gam, int N) {
    const float4 xk = xs4[k];
    float fx = 0.0f, fy = 0.0f, fz = 0.0f;
    if (!gamma_matrix(N)) {
        for (int j = 0; j < N; ++j) {
            if (j == k) continue;
            const int p = k < j ? pair_id(k, j, N) : pair_id(j, k, N);
            const float4 xj = xs4[j];
            const float dx = xk.x - xj.x, dy = xk.y - xj.y, dz = xk.z - xj.z;
            const float ir = rsqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
            const float c = gam[p] * ir * ir * ir;
            fx = fmaf(c, dx, fx);
            fy = fmaf(c, dy, fy);
            fz = fmaf(c, dz, fz);
        }
        return make_float3(fx, fy, fz);
    }
    const float* row = gam + k * gamma_stride(N);
    // x and y as one packed pair: d = x_k - x_j (a multiply by -1 is exact,
    // so the fused form rounds like the subtraction), f += c d
    float2 fxy = make_float2(0.0f, 0.0f);
    const float2 xky = make_float2(xk.x, xk.y), m1 = make_float2(-1.0f, -1.0f);
#pragma unroll 5
    for (int j = 0; j < N; ++j) {
        const float c = row[j];
        const float4 xj = xs4[j];
        const float2 d = __ffma2_rn(m1, make_float2(xj.x, xj.y), xky);
        fxy = __ffma2_rn(make_float2(c, c), d, fxy);
        fz = fmaf(c, xk.z - xj.z, fz);
    }
    return make_float3(fxy.x, fxy.y, fz);
}

// the terms j0 <= j < j1 of atom_force4's matrix-form sum (same arithmetic)
__device__ __forceinline__ float3 atom_force4_range(int k, const float4* xs4, const float* gam, int N, int j0,
                                                    int j1) {
    const float4 xk = xs4[k];
    const float* row = gam + k * gamma_stride(N);
    float2 fxy = make_float2(0.0f, 0.0f);
    float fz = 0.0f;
    const float2 xky = make_float2(xk.x, xk.y), m1 = make_float2(-1.0f, -1.0f);
#pragma unroll 5
    for (int j = j0; j < j1; ++j) {
        const float c = row[j];
        const float4 xj = xs4[j];
        const float2 d = __ffma2_rn(m1, make_float2(xj.x, xj.y), xky);
        fxy = __ffma2_rn(make_float2(c, c), d, fxy);
        fz = fmaf(c, xk.z - xj.z, fz);
    }
    return make_float3(fxy.x, fxy.y, fz);
}

// normalised energy e = b3 + sum of the layer-2 partial sums
__device__ __forceinline__ double head_energy(const float* part, int nparts, int m, const float* b3) {
    double e = (double)*b3;
    for (int q = 0; q < nparts; ++q) e += (double)part[(size_t)m * nparts + q];
    return e;
}

// sum of v over the block (blockDim.x a multiple of 32, <= 1024); every
// thread receives the total.  red: >= 32 doubles of shared memory.
__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < nw; ++i) t += red[i];
    return t;
}

}  // namespace pamd
