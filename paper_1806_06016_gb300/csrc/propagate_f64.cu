// propagate_f64.cu -- all-FP64 mode (PAMD_PREC_FP64): the same method with
// every quantity in binary64 on the GPU, as a precision reference for the
// mixed FP32/FP64 kernels.
//
// Layout: replica state [R][6][Np] doubles.  One warp advances one replica at
// a time; lane l owns atoms l, l+32, ...  Nonbonded forces are summed over
// all j for each owned atom (no Newton's third law: plain and obviously
// symmetric), bonded terms are spread over the lanes and added to per-atom
// shared-memory accumulators with atomicAdd.  Noise, init and resampling use
// the same Philox counters as the mixed path, Box-Muller in double.
#include <math.h>

#include "pamd_device.cuh"
#include "pamd_internal.h"

namespace pamd {

namespace {

constexpr int kF64Warps = 4;

__device__ __forceinline__ double u23d(uint32_t u) { return ((double)(u >> 9) + 0.5) * 0x1p-23; }

__device__ __forceinline__ void normal3d(unsigned long long seed, uint32_t atom, uint32_t slot,
                                         uint32_t step, uint32_t purpose, double z[3]) {
    const uint4 o = philox4x32_10(make_uint4(atom, slot, step, purpose), seed_key(seed));
    const double two_pi = 6.283185307179586476925286766559;
    const double r0 = sqrt(-2.0 * log(u23d(o.x)));
    const double r1 = sqrt(-2.0 * log(u23d(o.z)));
    z[0] = r0 * cos(two_pi * u23d(o.y));
    z[1] = r0 * sin(two_pi * u23d(o.y));
    z[2] = r1 * cos(two_pi * u23d(o.w));
}

struct D3 {
    double x, y, z;
};
__device__ __forceinline__ D3 dsub(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ double ddot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ D3 dcross(D3 a, D3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

__device__ __forceinline__ D3 ldpos(const double4* pos, int i) {
    const double4 p = pos[i];
    return {p.x, p.y, p.z};
}
__device__ __forceinline__ void addf(double4* frc, int i, D3 f) {
    atomicAdd(&frc[i].x, f.x);
    atomicAdd(&frc[i].y, f.y);
    atomicAdd(&frc[i].z, f.z);
}

// Bonded terms, lanes striding over each list; forces into frc (shared
// memory, atomics), energy into e.
template <bool ENERGY>
__device__ void bonded_f64(const TopoF64& t, const double4* pos, double4* frc, int lane,
                           double& e) {
    for (int b = lane; b < t.n_bonds; b += 32) {
        const int i = t.bond[2 * b], j = t.bond[2 * b + 1];
        const D3 d = dsub(ldpos(pos, i), ldpos(pos, j));
        const double r = sqrt(ddot(d, d));
        const double r0 = t.bond_p[2 * b], k = t.bond_p[2 * b + 1];
        if (ENERGY) e += 0.5 * k * (r - r0) * (r - r0);
        else {
            const double g = (r0 == 0.0) ? k : k * (r - r0) / r;
            addf(frc, i, {-g * d.x, -g * d.y, -g * d.z});
            addf(frc, j, {g * d.x, g * d.y, g * d.z});
        }
    }
    for (int a = lane; a < t.n_angles; a += 32) {
        const int i = t.angle[3 * a], j = t.angle[3 * a + 1], k = t.angle[3 * a + 2];
        const D3 u = dsub(ldpos(pos, i), ldpos(pos, j));
        const D3 w = dsub(ldpos(pos, k), ldpos(pos, j));
        const D3 uxw = dcross(u, w);
        const double s = sqrt(ddot(uxw, uxw)), c = ddot(u, w);
        const double dth = atan2(s, c) - t.angle_p[2 * a];
        const double kk = t.angle_p[2 * a + 1];
        if (ENERGY) e += 0.5 * kk * dth * dth;
        else {
            const double g = kk * dth, uu = ddot(u, u), ww = ddot(w, w);
            const D3 fi = {g * (w.x - c * u.x / uu) / s, g * (w.y - c * u.y / uu) / s,
                           g * (w.z - c * u.z / uu) / s};
            const D3 fk = {g * (u.x - c * w.x / ww) / s, g * (u.y - c * w.y / ww) / s,
                           g * (u.z - c * w.z / ww) / s};
            addf(frc, i, fi);
            addf(frc, k, fk);
            addf(frc, j, {-fi.x - fk.x, -fi.y - fk.y, -fi.z - fk.z});
        }
    }
    for (int h = lane; h < t.n_dihs; h += 32) {
        const int i = t.dih[4 * h], j = t.dih[4 * h + 1], k = t.dih[4 * h + 2], l = t.dih[4 * h + 3];
        const double kd = t.dih_p[4 * h], nn = t.dih_p[4 * h + 1];
        const double cph = t.dih_p[4 * h + 2], sph = t.dih_p[4 * h + 3];
        const D3 F = dsub(ldpos(pos, i), ldpos(pos, j));
        const D3 G = dsub(ldpos(pos, j), ldpos(pos, k));
        const D3 H = dsub(ldpos(pos, l), ldpos(pos, k));
        const D3 A = dcross(F, G), Bv = dcross(H, G);
        const double AA = ddot(A, A), BB = ddot(Bv, Bv), lg = sqrt(ddot(G, G));
        const double phi = atan2(ddot(dcross(Bv, A), G) / lg, ddot(A, Bv));
        if (ENERGY) e += kd * (1.0 + cos(nn * phi) * cph + sin(nn * phi) * sph);
        else {
            const double dEdphi = -kd * nn * (sin(nn * phi) * cph - cos(nn * phi) * sph);
            const double ia = lg / AA, ib = lg / BB;
            const double pa = ddot(F, G) / (AA * lg), pb = ddot(H, G) / (BB * lg);
            addf(frc, i, {dEdphi * ia * A.x, dEdphi * ia * A.y, dEdphi * ia * A.z});
            addf(frc, l, {-dEdphi * ib * Bv.x, -dEdphi * ib * Bv.y, -dEdphi * ib * Bv.z});
            const double ja = -dEdphi * (ia + pa), jb = dEdphi * pb;
            const double ka = dEdphi * pa, kb = -dEdphi * (pb - ib);
            addf(frc, j, {ja * A.x + jb * Bv.x, ja * A.y + jb * Bv.y, ja * A.z + jb * Bv.z});
            addf(frc, k, {ka * A.x + kb * Bv.x, ka * A.y + kb * Bv.y, ka * A.z + kb * Bv.z});
        }
    }
}

// Nonbonded pair (i, j) with scale factors; returns the force on i and adds
// the pair energy to e.
__device__ __forceinline__ D3 nb_pair_f64(const TopoF64& t, D3 xi, D3 xj, int i, int j, double slj,
                                          double sc, double& e) {
    const D3 d = dsub(xi, xj);
    const double r2 = ddot(d, d), r = sqrt(r2);
    const double sig = t.sigma_half[i] + t.sigma_half[j];
    const double eps = sqrt(t.epsilon[i] * t.epsilon[j]);
    const double sr2 = sig * sig / r2, sr6 = sr2 * sr2 * sr2, sr12 = sr6 * sr6;
    const double qq = kCoulomb * t.charge[i] * t.charge[j];
    e += slj * 4.0 * eps * (sr12 - sr6) + sc * qq / r;
    const double g = slj * 24.0 * eps * (2.0 * sr12 - sr6) / r2 + sc * qq / (r2 * r);
    return {g * d.x, g * d.y, g * d.z};
}

// A = ceil(N / 32) atoms per lane.  Dynamic shared memory: per warp N double4
// positions and N double4 bonded-force accumulators.
template <int A>
__global__ void __launch_bounds__(kF64Warps * 32) propagate_f64_kernel(PropF64Params p) {
    constexpr int kF64MaxPerLane = A;
    extern __shared__ double4 smem_d4[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const TopoF64& t = p.top;
    const int N = t.n_atoms, Np = p.n_pad;
    double4* pos = smem_d4 + (size_t)w * 2 * N;
    double4* frc = pos + N;
    const uint32_t step_base = (p.dev_counters ? p.dev_counters[0] : 0u) + p.step0;
    const double c1 = exp(-p.gamma * p.dt), c2kT = sqrt((1.0 - c1 * c1) * kBoltzmann * p.T);
    const double hdt = 0.5 * p.dt;
    for (long long k = (long long)blockIdx.x * kF64Warps + w; k < p.R;
         k += (long long)gridDim.x * kF64Warps) {
        double* st = p.state + (size_t)k * 6 * Np;
        D3 x[kF64MaxPerLane], v[kF64MaxPerLane], f[kF64MaxPerLane];
#pragma unroll
        for (int a = 0; a < kF64MaxPerLane; ++a) {
            const int i = lane + 32 * a;
            if (i < N) {
                x[a] = {st[i], st[Np + i], st[2 * Np + i]};
                v[a] = {st[3 * Np + i], st[4 * Np + i], st[5 * Np + i]};
                pos[i] = make_double4(x[a].x, x[a].y, x[a].z, 0.0);
            }
        }
        // s = -1 evaluates the forces of the incoming state
        for (int s = -1; s < p.theta; ++s) {
            if (s >= 0) {
                const uint32_t step = step_base + (uint32_t)s;
#pragma unroll
                for (int a = 0; a < kF64MaxPerLane; ++a) {
                    const int i = lane + 32 * a;
                    if (i >= N) continue;
                    const double im = t.inv_mass[i];
                    const double sd = c2kT * sqrt(im);
                    double z[3];
                    normal3d(p.seed, (uint32_t)i, (uint32_t)k, step, p.purpose_mol, z);
                    v[a].x += hdt * f[a].x * im; v[a].y += hdt * f[a].y * im; v[a].z += hdt * f[a].z * im;
                    x[a].x += hdt * v[a].x; x[a].y += hdt * v[a].y; x[a].z += hdt * v[a].z;
                    v[a].x = c1 * v[a].x + sd * z[0];
                    v[a].y = c1 * v[a].y + sd * z[1];
                    v[a].z = c1 * v[a].z + sd * z[2];
                    x[a].x += hdt * v[a].x; x[a].y += hdt * v[a].y; x[a].z += hdt * v[a].z;
                    pos[i] = make_double4(x[a].x, x[a].y, x[a].z, 0.0);
                }
            }
            for (int i = lane; i < N; i += 32) frc[i] = make_double4(0.0, 0.0, 0.0, 0.0);
            __syncwarp();
            double e_unused = 0.0;
            bonded_f64<false>(t, pos, frc, lane, e_unused);
#pragma unroll
            for (int a = 0; a < kF64MaxPerLane; ++a) {
                const int i = lane + 32 * a;
                if (i >= N) continue;
                D3 acc = {0.0, 0.0, 0.0};
                for (int j = 0; j < N; ++j) {
                    if (j == i) continue;
                    const unsigned char kind = t.kind[i * N + j];
                    if (kind == 1) continue;
                    const double slj = kind == 2 ? t.s14_lj : 1.0, sc = kind == 2 ? t.s14_c : 1.0;
                    const D3 fij = nb_pair_f64(t, x[a], ldpos(pos, j), i, j, slj, sc, e_unused);
                    acc.x += fij.x; acc.y += fij.y; acc.z += fij.z;
                }
                f[a] = acc;
            }
            __syncwarp();
#pragma unroll
            for (int a = 0; a < kF64MaxPerLane; ++a) {
                const int i = lane + 32 * a;
                if (i >= N) continue;
                const double4 b = frc[i];
                f[a].x += b.x; f[a].y += b.y; f[a].z += b.z;
                if (s >= 0) {
                    const double im = t.inv_mass[i];
                    v[a].x += hdt * f[a].x * im; v[a].y += hdt * f[a].y * im; v[a].z += hdt * f[a].z * im;
                }
            }
            __syncwarp();
        }
        // energy (pairs j > i counted once) and per-replica observables
        double e = 0.0;
        bonded_f64<true>(t, pos, frc, lane, e);
        double ek = 0.0, cx = 0.0, cy = 0.0, cz = 0.0;
#pragma unroll
        for (int a = 0; a < kF64MaxPerLane; ++a) {
            const int i = lane + 32 * a;
            if (i >= N) continue;
            for (int j = i + 1; j < N; ++j) {
                const unsigned char kind = t.kind[i * N + j];
                if (kind == 1) continue;
                const double slj = kind == 2 ? t.s14_lj : 1.0, sc = kind == 2 ? t.s14_c : 1.0;
                nb_pair_f64(t, x[a], ldpos(pos, j), i, j, slj, sc, e);
            }
            if (p.theta > 0) {
                st[i] = x[a].x; st[Np + i] = x[a].y; st[2 * Np + i] = x[a].z;
                st[3 * Np + i] = v[a].x; st[4 * Np + i] = v[a].y; st[5 * Np + i] = v[a].z;
            }
            if (p.fout) {
                double* fo = p.fout + (size_t)k * 3 * Np;
                fo[i] = f[a].x; fo[Np + i] = f[a].y; fo[2 * Np + i] = f[a].z;
            }
            ek += 0.5 * (1.0 / t.inv_mass[i]) * ddot(v[a], v[a]);
            cx += x[a].x; cy += x[a].y; cz += x[a].z;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            e += __shfl_xor_sync(0xffffffffu, e, o);
            ek += __shfl_xor_sync(0xffffffffu, ek, o);
            cx += __shfl_xor_sync(0xffffffffu, cx, o);
            cy += __shfl_xor_sync(0xffffffffu, cy, o);
            cz += __shfl_xor_sync(0xffffffffu, cz, o);
        }
        cx /= N; cy /= N; cz /= N;
        double r2 = 0.0;
#pragma unroll
        for (int a = 0; a < kF64MaxPerLane; ++a) {
            const int i = lane + 32 * a;
            if (i >= N) continue;
            const double dx = x[a].x - cx, dy = x[a].y - cy, dz = x[a].z - cz;
            r2 += dx * dx + dy * dy + dz * dz;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
        if (lane == 0) {
            p.E[k] = e;
            p.ke[k] = ek;
            p.rg[k] = sqrt(r2 / N);
            if (!isfinite(e) && atomicCAS(&p.status[0], 0, PAMD_ENONFINITE) == 0) p.status[1] = (int)k;
        }
        __syncwarp();
    }
}

__global__ void init_f64_kernel(double* state, double* E, int32_t* fam, const double* x0,
                                const double* inv_mass, long long R, int N, int Np, double kT0,
                                unsigned long long seed, uint32_t purpose) {
    const long long total = R * (long long)Np;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long k = t / Np;
        const int i = (int)(t - k * Np);
        double* st = state + (size_t)k * 6 * Np;
        if (i < N) {
            double z[3];
            normal3d(seed, (uint32_t)i, (uint32_t)k, 0u, purpose, z);
            const double sdv = sqrt(kT0 * inv_mass[i]);
            st[i] = x0[i];
            st[Np + i] = x0[Np + i];
            st[2 * Np + i] = x0[2 * Np + i];
            st[3 * Np + i] = sdv * z[0];
            st[4 * Np + i] = sdv * z[1];
            st[5 * Np + i] = sdv * z[2];
        } else {
#pragma unroll
            for (int c = 0; c < 6; ++c) st[c * Np + i] = 0.0;
        }
        if (i == 0) {
            fam[k] = (int32_t)k;
            E[k] = 0.0;
        }
    }
}

// One warp per new slot k, ancestor by binary search of the inclusive counts;
// positions recentred on the centre of mass, velocities scaled.
__global__ void gather_f64_kernel(const double* __restrict__ st_in, double* __restrict__ st_out,
                                  const double* E_in, double* E_out, const int32_t* fam_in,
                                  int32_t* fam_out, double* ke_out, double* rg_out,
                                  const int32_t* incl, const double* inv_mass, long long R, int N,
                                  int Np, double vscale) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long k = warp; k < R; k += nwarps) {
        long long lo = 0, hi = R;
        while (lo < hi) {
            const long long mid = lo + ((hi - lo) >> 1);
            if (incl[mid] > k) hi = mid;
            else lo = mid + 1;
        }
        const long long j = lo < R ? lo : R - 1;
        const double* src = st_in + (size_t)j * 6 * Np;
        double* dst = st_out + (size_t)k * 6 * Np;
        double m = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
        for (int i = lane; i < N; i += 32) {
            const double mi = 1.0 / inv_mass[i];
            m += mi;
            sx += mi * src[i];
            sy += mi * src[Np + i];
            sz += mi * src[2 * Np + i];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            m += __shfl_xor_sync(0xffffffffu, m, o);
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
            sz += __shfl_xor_sync(0xffffffffu, sz, o);
        }
        const double cx = sx / m, cy = sy / m, cz = sz / m;
        double mv2 = 0.0, ux = 0.0, uy = 0.0, uz = 0.0, u2 = 0.0;
        for (int i = lane; i < Np; i += 32) {
            if (i < N) {
                const double x = src[i] - cx, y = src[Np + i] - cy, z = src[2 * Np + i] - cz;
                const double vx = vscale * src[3 * Np + i], vy = vscale * src[4 * Np + i],
                             vz = vscale * src[5 * Np + i];
                dst[i] = x; dst[Np + i] = y; dst[2 * Np + i] = z;
                dst[3 * Np + i] = vx; dst[4 * Np + i] = vy; dst[5 * Np + i] = vz;
                mv2 += (vx * vx + vy * vy + vz * vz) / inv_mass[i];
                ux += x; uy += y; uz += z;
                u2 += x * x + y * y + z * z;
            } else {
#pragma unroll
                for (int c = 0; c < 6; ++c) dst[c * Np + i] = 0.0;
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
            ke_out[k] = 0.5 * mv2;
            const double mx = ux / N, my = uy / N, mz = uz / N;
            rg_out[k] = sqrt(fmax(u2 / N - (mx * mx + my * my + mz * mz), 0.0));
        }
    }
}

}  // namespace

cudaError_t launch_propagate_f64(pamd_ctx* c, double* state, double* E, double* ke, double* rg,
                                 int theta, double dt, double T, const uint32_t* dev_ctr,
                                 uint32_t step0, double* fout) {
    PropF64Params p{};
    p.state = state;
    p.E = E;
    p.ke = ke;
    p.rg = rg;
    p.fout = fout;
    p.status = &c->b.scal->status;
    p.dev_counters = dev_ctr;
    p.top = c->top64;
    p.n_pad = c->Np;
    p.R = c->R;
    p.theta = theta;
    p.dt = dt;
    p.T = T;
    p.gamma = c->gamma;
    p.seed = c->seed;
    p.step0 = step0;
    p.purpose_mol = kPurposeNoise | ((uint32_t)c->mol << 8);
    const long long blocks = (c->R + kF64Warps - 1) / kF64Warps;
    const int grid = (int)(blocks < (long long)c->num_sms * 8 ? blocks : (long long)c->num_sms * 8);
    const size_t smem = (size_t)kF64Warps * 2 * c->N * sizeof(double4);
    cudaError_t e = cudaSuccess;
    switch ((c->N + 31) / 32) {
#define PAMD_F64_CASE(A)                                                                          \
    case A:                                                                                       \
        e = cudaFuncSetAttribute(propagate_f64_kernel<A>,                                         \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);         \
        if (e == cudaSuccess) propagate_f64_kernel<A><<<grid, kF64Warps * 32, smem, c->stream>>>(p); \
        break;
        PAMD_F64_CASE(1) PAMD_F64_CASE(2) PAMD_F64_CASE(3) PAMD_F64_CASE(4)
        PAMD_F64_CASE(5) PAMD_F64_CASE(6) PAMD_F64_CASE(7) PAMD_F64_CASE(8)
#undef PAMD_F64_CASE
        default: return cudaErrorInvalidValue;
    }
    c->launches += 1;
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_init_f64(pamd_ctx* c, double T0) {
    const long long total = c->R * c->Np;
    long long g = (total + 255) / 256;
    if (g > (long long)c->num_sms * 16) g = (long long)c->num_sms * 16;
    init_f64_kernel<<<(int)g, 256, 0, c->stream>>>(
        reinterpret_cast<double*>(c->b.state), c->b.E, c->b.fam, c->top64.x0, c->top64.inv_mass,
        c->R, c->N, c->Np, kBoltzmann * T0, c->seed, kPurposeInit | ((uint32_t)c->mol << 8));
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_gather_f64(pamd_ctx* c, const double* src, double* dst, const double* Ein,
                              double* Eout, const int32_t* fin, int32_t* fout, double vscale) {
    long long g = (c->R * 32 + 255) / 256;
    if (g > (long long)c->num_sms * 32) g = (long long)c->num_sms * 32;
    gather_f64_kernel<<<(int)g, 256, 0, c->stream>>>(src, dst, Ein, Eout, fin, fout, c->b.ke,
                                                       c->b.rg, c->b.cnt_incl, c->top64.inv_mass,
                                                       c->R, c->N, c->Np, vscale);
    c->launches += 1;
    return cudaGetLastError();
}

}  // namespace pamd
