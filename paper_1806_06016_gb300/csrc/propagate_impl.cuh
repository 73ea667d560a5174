// propagate_impl.cuh -- persistent BAOAB Langevin kernel (PAMD scheme, step 3).
//
// Mapping.  A replica is owned by a group of L lanes of one warp (L = 4, 8,
// 16 or 32; 32/L replicas per warp).  Lane g of the group owns the B atoms
// [g*B, g*B+B) of the molecule: their positions, velocities, parameters and
// force accumulators live in registers for all theta steps.  Positions are
// mirrored to shared memory (one float4 per atom) so that other lanes can read
// them, and a float4 per atom in shared memory collects force contributions
// written by other lanes.
//
// Nonbonded forces use Newton's third law over a "half ring" of lane blocks:
// at step t (1 <= t <= L/2) lane g pairs its block with block (g+t) mod L
// (at t = L/2 only lanes g < L/2 do, so that the antipodal pair is done once),
// accumulating its own atoms' forces in registers and the partner block's in
// registers that are then added to shared memory.  At each t the partner
// blocks of the lanes are distinct, so those read-modify-writes need no
// atomics; a __syncwarp separates the steps.  The block's internal pairs
// (t = 0) are done by the owner.  Pairs that the topology excludes or scales
// (1-2, 1-3, 1-4) are masked out of their tile by a 64-bit mask per tile;
// 1-4 pairs are then added with their scale factors in the bonded pass.
// Bonded terms are split into colour classes whose terms share no atom, so
// all lanes of the group can add their forces without atomics.
//
// Atoms beyond N (padding up to L*B) get zero parameters, infinite mass and
// positions 1000 nm away from everything, so they contribute exactly zero.
#pragma once

#include "pamd_device.cuh"
#include "pamd_internal.h"

namespace pamd {

template <int L, int B>
struct PropCfg {
    static constexpr int BS = (B % 2 == 1) ? B : B + 1;  // odd stride: conflict-free LDS.128
    static constexpr int NK = L * BS;                     // shared-memory atom slots
    static constexpr int TH = L / 2;                      // half-ring steps
    static constexpr int SLOT = 2 * NK + 1;               // float4s per replica slot (pos + frc + pad)
};

// Lennard-Jones + Coulomb for one pair.  d = x_j - x_i.  With
// eps = 24 sqrt(eps_i eps_j) and qq = k_e q_i q_j the force on i is -fs * d
// and on j +fs * d; e is 4 eps_ij [(s/r)^12 - (s/r)^6] + k_e q_i q_j / r.
template <bool ENERGY>
__device__ __forceinline__ void pair_lj_coul(float dx, float dy, float dz, float sig, float eps,
                                             float qq, float& fs, float& e) {
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float rinv = rsqrtf(r2);
    const float rinv2 = rinv * rinv;
    const float s2 = sig * sig * rinv2;
    const float s6 = s2 * s2 * s2;
    const float lj = eps * s6 * fmaf(2.0f, s6, -1.0f);
    const float cq = qq * rinv;
    fs = (lj + cq) * rinv2;
    if (ENERGY) e = fmaf((eps * (1.0f / 6.0f)) * s6, s6 - 1.0f, cq);
}

template <int B, bool MASKED, bool ENERGY>
__device__ __forceinline__ void pair_tile(const float (&xi)[B], const float (&yi)[B],
                                          const float (&zi)[B], const float (&hsi)[B],
                                          const float (&sei)[B], const float (&qi)[B],
                                          float (&fxi)[B], float (&fyi)[B], float (&fzi)[B],
                                          const float4 (&pj)[B], const float4 (&cj)[B],
                                          float (&fxj)[B], float (&fyj)[B], float (&fzj)[B],
                                          unsigned long long mask, double& e_acc) {
#pragma unroll
    for (int a = 0; a < B; ++a) {
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const float dx = pj[b].x - xi[a];
            const float dy = pj[b].y - yi[a];
            const float dz = pj[b].z - zi[a];
            float fs, e;
            pair_lj_coul<ENERGY>(dx, dy, dz, hsi[a] + cj[b].x, sei[a] * cj[b].y, qi[a] * cj[b].z,
                                 fs, e);
            if (MASKED) {
                const bool skip = (mask >> (a * B + b)) & 1ull;
                fs = skip ? 0.0f : fs;
                if (ENERGY) e = skip ? 0.0f : e;
            }
            fxi[a] = fmaf(-fs, dx, fxi[a]);
            fyi[a] = fmaf(-fs, dy, fyi[a]);
            fzi[a] = fmaf(-fs, dz, fzi[a]);
            fxj[b] = fmaf(fs, dx, fxj[b]);
            fyj[b] = fmaf(fs, dy, fyj[b]);
            fzj[b] = fmaf(fs, dz, fzj[b]);
            if (ENERGY) e_acc += (double)e;
        }
    }
}

__device__ __forceinline__ void add_force(float4* frc, int s, float fx, float fy, float fz) {
    float4 f = frc[s];
    f.x += fx;
    f.y += fy;
    f.z += fz;
    frc[s] = f;
}

__device__ __forceinline__ float3 sub3(float4 a, float4 b) {
    return make_float3(a.x - b.x, a.y - b.y, a.z - b.z);
}
__device__ __forceinline__ float dot3(float3 a, float3 b) {
    return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z));
}
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// Bonded terms and scaled 1-4 pairs: colour by colour, lanes of the group
// stride over the terms of a colour.
template <int L, bool ENERGY>
__device__ __forceinline__ void bonded_forces(const unsigned char* sm, const TopoLayout& lay,
                                              const float4* prm, const float4* pos, float4* frc,
                                              int g, unsigned gmask, double& e_acc) {
    const int* colors = reinterpret_cast<const int*>(sm + lay.off_colors);
    // bonds: 1/2 k (r - r0)^2
    {
        const BondRec* rec = reinterpret_cast<const BondRec*>(sm + lay.off_bonds);
        const int* cs = colors + 0 * (kMaxColors + 1);
        for (int c = 0; c < lay.n_colors[0]; ++c) {
            for (int t = cs[c] + g; t < cs[c + 1]; t += L) {
                const BondRec b = rec[t];
                const float3 d = sub3(pos[b.i], pos[b.j]);
                const float r2 = dot3(d, d);
                const float r = sqrtf(r2);
                const float gk = (b.r0 == 0.0f) ? b.k : b.k * (r - b.r0) / r;
                add_force(frc, b.i, -gk * d.x, -gk * d.y, -gk * d.z);
                add_force(frc, b.j, gk * d.x, gk * d.y, gk * d.z);
                if (ENERGY) e_acc += (double)(0.5f * b.k * (r - b.r0) * (r - b.r0));
            }
            __syncwarp(gmask);
        }
    }
    // angles: 1/2 k (theta - theta0)^2
    {
        const AngleRec* rec = reinterpret_cast<const AngleRec*>(sm + lay.off_angles);
        const int* cs = colors + 1 * (kMaxColors + 1);
        for (int c = 0; c < lay.n_colors[1]; ++c) {
            for (int t = cs[c] + g; t < cs[c + 1]; t += L) {
                const AngleRec a = rec[t];
                const float3 u = sub3(pos[a.i], pos[a.j]);
                const float3 w = sub3(pos[a.k], pos[a.j]);
                const float3 uxw = cross3(u, w);
                const float s = sqrtf(dot3(uxw, uxw));
                const float cw = dot3(u, w);
                const float th = atan2f(s, cw);
                const float dth = th - a.t0;
                const float gk = a.kk * dth;
                const float is = 1.0f / s;
                const float cu = cw / dot3(u, u), cv = cw / dot3(w, w);
                // dtheta/du = -(w - (u.w) u/|u|^2)/|u x w|, dtheta/dw likewise
                const float3 du = make_float3(-(w.x - cu * u.x) * is, -(w.y - cu * u.y) * is,
                                              -(w.z - cu * u.z) * is);
                const float3 dw = make_float3(-(u.x - cv * w.x) * is, -(u.y - cv * w.y) * is,
                                              -(u.z - cv * w.z) * is);
                add_force(frc, a.i, -gk * du.x, -gk * du.y, -gk * du.z);
                add_force(frc, a.k, -gk * dw.x, -gk * dw.y, -gk * dw.z);
                add_force(frc, a.j, gk * (du.x + dw.x), gk * (du.y + dw.y), gk * (du.z + dw.z));
                if (ENERGY) e_acc += (double)(0.5f * a.kk * dth * dth);
            }
            __syncwarp(gmask);
        }
    }
    // dihedrals: k (1 + cos(n phi - phase)), gradient after Blondel & Karplus (1996)
    {
        const DihRec* rec = reinterpret_cast<const DihRec*>(sm + lay.off_dihs);
        const int* cs = colors + 2 * (kMaxColors + 1);
        for (int c = 0; c < lay.n_colors[2]; ++c) {
            for (int t = cs[c] + g; t < cs[c + 1]; t += L) {
                const DihRec h = rec[t];
                const float4 pi_ = pos[h.i], pj_ = pos[h.j], pk_ = pos[h.k], pl_ = pos[h.l];
                const float3 F = sub3(pi_, pj_);
                const float3 G = sub3(pj_, pk_);
                const float3 H = sub3(pl_, pk_);
                const float3 A = cross3(F, G);
                const float3 Bv = cross3(H, G);
                const float AA = dot3(A, A), BB = dot3(Bv, Bv);
                const float lg = sqrtf(dot3(G, G));
                const float rab = rsqrtf(AA * BB);
                const float cphi = dot3(A, Bv) * rab;
                const float sphi = dot3(cross3(Bv, A), G) * rab / lg;
                // cos(n phi), sin(n phi) by the angle-addition recurrence
                float cn = cphi, sn = sphi;
                const int n = (int)h.n;
                for (int q = 1; q < n; ++q) {
                    const float c2 = cn * cphi - sn * sphi;
                    sn = sn * cphi + cn * sphi;
                    cn = c2;
                }
                // dE/dphi = -k n sin(n phi - phase)
                const float sdel = sn * h.cos_ph - cn * h.sin_ph;
                const float dEdphi = -h.kd * h.n * sdel;
                const float fg = dot3(F, G), hg = dot3(H, G);
                const float ia = lg / AA, ib = lg / BB;
                const float pa = fg / (AA * lg), pb = hg / (BB * lg);
                // F_atom = -dE/dphi * dphi/dx_atom
                const float ci = dEdphi * ia;           // dphi/dx_i = -ia A
                const float cl = -dEdphi * ib;          // dphi/dx_l = +ib B
                add_force(frc, h.i, ci * A.x, ci * A.y, ci * A.z);
                add_force(frc, h.l, cl * Bv.x, cl * Bv.y, cl * Bv.z);
                // dphi/dx_j = (ia + pa) A - pb B ; dphi/dx_k = -pa A + (pb - ib) B
                const float ja = -dEdphi * (ia + pa), jb = dEdphi * pb;
                const float ka = dEdphi * pa, kb = -dEdphi * (pb - ib);
                add_force(frc, h.j, ja * A.x + jb * Bv.x, ja * A.y + jb * Bv.y, ja * A.z + jb * Bv.z);
                add_force(frc, h.k, ka * A.x + kb * Bv.x, ka * A.y + kb * Bv.y, ka * A.z + kb * Bv.z);
                if (ENERGY) {
                    const float cdel = cn * h.cos_ph + sn * h.sin_ph;
                    e_acc += (double)(h.kd * (1.0f + cdel));
                }
            }
            __syncwarp(gmask);
        }
    }
    // 1-4 pairs with scaled Lennard-Jones and Coulomb
    {
        const Pair14Rec* rec = reinterpret_cast<const Pair14Rec*>(sm + lay.off_p14);
        const int* cs = colors + 3 * (kMaxColors + 1);
        for (int c = 0; c < lay.n_colors[3]; ++c) {
            for (int t = cs[c] + g; t < cs[c + 1]; t += L) {
                const Pair14Rec q = rec[t];
                const float4 ci = prm[q.i], cj = prm[q.j];
                const float3 d = sub3(pos[q.j], pos[q.i]);
                const float r2 = dot3(d, d);
                const float rinv = rsqrtf(r2);
                const float rinv2 = rinv * rinv;
                const float sig = ci.x + cj.x;
                const float s2 = sig * sig * rinv2;
                const float s6 = s2 * s2 * s2;
                const float eps = ci.y * cj.y;
                const float cq = q.s_c * ci.z * cj.z * rinv;
                const float lj = q.s_lj * eps * s6 * fmaf(2.0f, s6, -1.0f);
                const float fs = (lj + cq) * rinv2;
                add_force(frc, q.i, -fs * d.x, -fs * d.y, -fs * d.z);
                add_force(frc, q.j, fs * d.x, fs * d.y, fs * d.z);
                if (ENERGY)
                    e_acc += (double)(q.s_lj * (eps * (1.0f / 6.0f)) * s6 * (s6 - 1.0f) + cq);
            }
            __syncwarp(gmask);
        }
    }
}

// Forces on the lane's B atoms (registers fx, fy, fz); positions must already
// be in shared memory and the lane's force slots zeroed, with a __syncwarp
// after both.
template <int L, int B, bool ENERGY>
__device__ __forceinline__ void compute_forces(const unsigned char* sm, const TopoLayout& lay,
                                               const float4* prm, const float4* pos, float4* frc,
                                               const unsigned long long* masks, int g,
                                               unsigned gmask, const float (&xi)[B],
                                               const float (&yi)[B], const float (&zi)[B],
                                               const float (&hsi)[B], const float (&sei)[B],
                                               const float (&qi)[B], float (&fx)[B],
                                               float (&fy)[B], float (&fz)[B], double& e_acc) {
    using C = PropCfg<L, B>;
#pragma unroll
    for (int a = 0; a < B; ++a) fx[a] = fy[a] = fz[a] = 0.0f;
    // pairs inside the lane's own block (always masked: 1-2/1-3/1-4 live here)
    {
        const unsigned long long m = masks[g];
#pragma unroll
        for (int a = 0; a < B; ++a) {
#pragma unroll
            for (int b = a + 1; b < B; ++b) {
                const float dx = xi[b] - xi[a], dy = yi[b] - yi[a], dz = zi[b] - zi[a];
                float fs, e;
                pair_lj_coul<ENERGY>(dx, dy, dz, hsi[a] + hsi[b], sei[a] * sei[b], qi[a] * qi[b],
                                     fs, e);
                const bool skip = (m >> (a * B + b)) & 1ull;
                fs = skip ? 0.0f : fs;
                fx[a] = fmaf(-fs, dx, fx[a]);
                fy[a] = fmaf(-fs, dy, fy[a]);
                fz[a] = fmaf(-fs, dz, fz[a]);
                fx[b] = fmaf(fs, dx, fx[b]);
                fy[b] = fmaf(fs, dy, fy[b]);
                fz[b] = fmaf(fs, dz, fz[b]);
                if (ENERGY) e_acc += skip ? 0.0 : (double)e;
            }
        }
    }
    // half ring over partner blocks
#pragma unroll 1
    for (int t = 1; t <= C::TH; ++t) {
        const bool active = (t < C::TH) || (g < C::TH);
        if (active) {
            const int J = (g + t) & (L - 1);
            float4 pj[B], cj[B];
            float fxj[B], fyj[B], fzj[B];
#pragma unroll
            for (int b = 0; b < B; ++b) {
                pj[b] = pos[J * C::BS + b];
                cj[b] = prm[J * C::BS + b];
                fxj[b] = fyj[b] = fzj[b] = 0.0f;
            }
            const unsigned long long m = masks[t * L + g];
            if (m == 0ull)
                pair_tile<B, false, ENERGY>(xi, yi, zi, hsi, sei, qi, fx, fy, fz, pj, cj, fxj, fyj,
                                            fzj, m, e_acc);
            else
                pair_tile<B, true, ENERGY>(xi, yi, zi, hsi, sei, qi, fx, fy, fz, pj, cj, fxj, fyj,
                                           fzj, m, e_acc);
#pragma unroll
            for (int b = 0; b < B; ++b) add_force(frc, J * C::BS + b, fxj[b], fyj[b], fzj[b]);
        }
        __syncwarp(gmask);
    }
    bonded_forces<L, ENERGY>(sm, lay, prm, pos, frc, g, gmask, e_acc);
#pragma unroll
    for (int a = 0; a < B; ++a) {
        const float4 f = frc[g * C::BS + a];
        fx[a] += f.x;
        fy[a] += f.y;
        fz[a] += f.z;
    }
}

template <int L>
__device__ __forceinline__ double group_sum(double v, unsigned gmask) {
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(gmask, v, o);
    return v;
}

template <int L, int B>
__global__ void __launch_bounds__(256, 1) propagate_kernel(const PropParams p) {
    using C = PropCfg<L, B>;
    extern __shared__ float4 smem4[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(smem4);
    const TopoLayout& lay = p.lay;
    {
        const float4* src = reinterpret_cast<const float4*>(p.topo);
        for (int i = threadIdx.x; i < lay.bytes / 16; i += blockDim.x) smem4[i] = src[i];
    }
    __syncthreads();
    const float4* prm = reinterpret_cast<const float4*>(sm + lay.off_params);
    const unsigned long long* masks = reinterpret_cast<const unsigned long long*>(sm + lay.off_masks);
    float4* slots = smem4 + lay.bytes / 16;

    const int lane = threadIdx.x & 31;
    const int grp = lane / L;
    const int g = lane % L;
    const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << (grp * L));
    const int groups_per_warp = 32 / L;
    const int slot_local = (threadIdx.x >> 5) * groups_per_warp + grp;
    const int rpb = (blockDim.x >> 5) * groups_per_warp;
    float4* pos = slots + slot_local * C::SLOT;
    float4* frc = pos + C::NK;

    const int N = lay.n_atoms, Np = lay.n_pad;
    const uint32_t step_base = (p.dev_counters ? p.dev_counters[0] : 0u) + p.step0;

    for (long long k = (long long)blockIdx.x * rpb + slot_local; k < p.R;
         k += (long long)gridDim.x * rpb) {
        const float* st = p.state_in + (size_t)k * 6 * Np;
        float xi[B], yi[B], zi[B], vx[B], vy[B], vz[B];
        float hsi[B], sei[B], qi[B], im[B], sd[B];
#pragma unroll
        for (int a = 0; a < B; ++a) {
            const int i = g * B + a;
            const int s = g * C::BS + a;
            if (i < N) {
                xi[a] = st[i];
                yi[a] = st[Np + i];
                zi[a] = st[2 * Np + i];
                vx[a] = st[3 * Np + i];
                vy[a] = st[4 * Np + i];
                vz[a] = st[5 * Np + i];
            } else {
                xi[a] = 1000.0f + 4.0f * (float)i;
                yi[a] = zi[a] = 0.0f;
                vx[a] = vy[a] = vz[a] = 0.0f;
            }
            const float4 c = prm[s];
            hsi[a] = c.x;
            sei[a] = c.y;
            qi[a] = c.z;
            im[a] = c.w;
            sd[a] = p.c2kT * sqrtf(c.w);
            pos[s] = make_float4(xi[a], yi[a], zi[a], 0.0f);
            frc[s] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
        __syncwarp(gmask);
        float fx[B], fy[B], fz[B];
        double e_acc = 0.0;
        if (p.theta == 0)
            compute_forces<L, B, true>(sm, lay, prm, pos, frc, masks, g, gmask, xi, yi, zi, hsi,
                                       sei, qi, fx, fy, fz, e_acc);
        else
            compute_forces<L, B, false>(sm, lay, prm, pos, frc, masks, g, gmask, xi, yi, zi, hsi,
                                        sei, qi, fx, fy, fz, e_acc);

        for (int s = 0; s < p.theta; ++s) {
            const uint32_t step = step_base + (uint32_t)s;
#pragma unroll
            for (int a = 0; a < B; ++a) {
                const int i = g * B + a;
                vx[a] = fmaf(p.hdt * im[a], fx[a], vx[a]);  // B
                vy[a] = fmaf(p.hdt * im[a], fy[a], vy[a]);
                vz[a] = fmaf(p.hdt * im[a], fz[a], vz[a]);
                xi[a] = fmaf(p.hdt, vx[a], xi[a]);          // A
                yi[a] = fmaf(p.hdt, vy[a], yi[a]);
                zi[a] = fmaf(p.hdt, vz[a], zi[a]);
                if (i < N) {                                // O
                    const float3 z = normal3(p.seed, (uint32_t)i, (uint32_t)k, step, p.purpose_mol);
                    vx[a] = fmaf(p.c1, vx[a], sd[a] * z.x);
                    vy[a] = fmaf(p.c1, vy[a], sd[a] * z.y);
                    vz[a] = fmaf(p.c1, vz[a], sd[a] * z.z);
                }
                xi[a] = fmaf(p.hdt, vx[a], xi[a]);          // A
                yi[a] = fmaf(p.hdt, vy[a], yi[a]);
                zi[a] = fmaf(p.hdt, vz[a], zi[a]);
                const int sl = g * C::BS + a;
                pos[sl] = make_float4(xi[a], yi[a], zi[a], 0.0f);
                frc[sl] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
            __syncwarp(gmask);
            if (s == p.theta - 1)
                compute_forces<L, B, true>(sm, lay, prm, pos, frc, masks, g, gmask, xi, yi, zi,
                                           hsi, sei, qi, fx, fy, fz, e_acc);
            else
                compute_forces<L, B, false>(sm, lay, prm, pos, frc, masks, g, gmask, xi, yi, zi,
                                            hsi, sei, qi, fx, fy, fz, e_acc);
#pragma unroll
            for (int a = 0; a < B; ++a) {                   // B
                vx[a] = fmaf(p.hdt * im[a], fx[a], vx[a]);
                vy[a] = fmaf(p.hdt * im[a], fy[a], vy[a]);
                vz[a] = fmaf(p.hdt * im[a], fz[a], vz[a]);
            }
        }

        // write back and per-replica observables
        float* so = p.state_out + (size_t)k * 6 * Np;
        double ek = 0.0, cx = 0.0, cy = 0.0, cz = 0.0;
#pragma unroll
        for (int a = 0; a < B; ++a) {
            const int i = g * B + a;
            if (i < N) {
                if (p.theta > 0) {
                    so[i] = xi[a];
                    so[Np + i] = yi[a];
                    so[2 * Np + i] = zi[a];
                    so[3 * Np + i] = vx[a];
                    so[4 * Np + i] = vy[a];
                    so[5 * Np + i] = vz[a];
                }
                if (p.fout) {
                    float* fo = p.fout + (size_t)k * 3 * Np;
                    fo[i] = fx[a];
                    fo[Np + i] = fy[a];
                    fo[2 * Np + i] = fz[a];
                }
                const double m = (double)p.masses[i];
                ek += 0.5 * m * ((double)vx[a] * vx[a] + (double)vy[a] * vy[a] + (double)vz[a] * vz[a]);
                cx += xi[a];
                cy += yi[a];
                cz += zi[a];
            }
        }
        const double E = group_sum<L>(e_acc, gmask);
        ek = group_sum<L>(ek, gmask);
        cx = group_sum<L>(cx, gmask) / N;
        cy = group_sum<L>(cy, gmask) / N;
        cz = group_sum<L>(cz, gmask) / N;
        double r2 = 0.0;
#pragma unroll
        for (int a = 0; a < B; ++a) {
            const int i = g * B + a;
            if (i < N) {
                const double dx = xi[a] - cx, dy = yi[a] - cy, dz = zi[a] - cz;
                r2 += dx * dx + dy * dy + dz * dz;
            }
        }
        r2 = group_sum<L>(r2, gmask);
        if (g == 0) {
            p.E[k] = E;
            p.ke[k] = ek;
            p.rg[k] = sqrt(r2 / N);
            if (!isfinite(E) && atomicCAS(&p.status[0], 0, PAMD_ENONFINITE) == 0)
                p.status[1] = (int)k;
        }
        __syncwarp(gmask);
    }
}

template <int L, int B>
cudaError_t propagate_launch_one(const PropParams* p, int warps, int grid, size_t smem,
                                 cudaStream_t s, int* blocks_per_sm) {
    auto kern = propagate_kernel<L, B>;
    static size_t configured = 0;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    if (!p) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, warps * 32, smem);
    kern<<<grid, warps * 32, smem, s>>>(*p);
    return cudaGetLastError();
}

template <int L>
cudaError_t propagate_dispatch(const PropParams* p, int per_lane, int warps, int grid, size_t smem,
                               cudaStream_t s, int* blocks_per_sm) {
    switch (per_lane) {
        case 1: return propagate_launch_one<L, 1>(p, warps, grid, smem, s, blocks_per_sm);
        case 2: return propagate_launch_one<L, 2>(p, warps, grid, smem, s, blocks_per_sm);
        case 3: return propagate_launch_one<L, 3>(p, warps, grid, smem, s, blocks_per_sm);
        case 4: return propagate_launch_one<L, 4>(p, warps, grid, smem, s, blocks_per_sm);
        case 5: return propagate_launch_one<L, 5>(p, warps, grid, smem, s, blocks_per_sm);
        case 6: return propagate_launch_one<L, 6>(p, warps, grid, smem, s, blocks_per_sm);
        case 7: return propagate_launch_one<L, 7>(p, warps, grid, smem, s, blocks_per_sm);
        case 8: return propagate_launch_one<L, 8>(p, warps, grid, smem, s, blocks_per_sm);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pamd
