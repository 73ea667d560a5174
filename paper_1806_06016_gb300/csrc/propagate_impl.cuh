// propagate_impl.cuh -- persistent BAOAB Langevin kernel (PAMD scheme, step 3).
//
// Mapping.  A replica is owned by a group of L lanes of one warp (1 <= L <= 32,
// G = floor(32/L) replicas per warp, the remaining 32 - G*L lanes idle).  Lane
// g of a group owns the B atoms [g*B, g*B+B) of the molecule: their
// positions, velocities, parameters and force accumulators live in registers
// for all theta steps.  Positions are mirrored to shared memory (one float4
// per atom) so that other lanes can read them, and a float4 per atom in
// shared memory collects force contributions written by other lanes.
//
// Nonbonded forces use Newton's third law over a "half ring" of lane blocks:
// at step t (1 <= t <= L/2) lane g pairs its block with block (g+t) mod L (for
// even L, at t = L/2 only lanes g < L/2 do, so the antipodal pair is done
// once), accumulating its own atoms' forces in registers and the partner
// block's in registers that are then added to shared memory.  At each t the
// partner blocks of the lanes are distinct, so those read-modify-writes need
// no atomics; a __syncwarp separates the steps.  The block's internal pairs
// (t = 0) are done by the owner.  Pairs that the topology excludes or scales
// (1-2, 1-3, 1-4) are masked out of their tile by a 64-bit mask per tile; 1-4
// pairs are then added with their scale factors in the bonded pass.
//
// Bonded terms.  For a linear chain (bonds (k,k+1), angles (k..k+2),
// dihedrals (k..k+3), 1-4 pairs (k,k+3)) each lane evaluates the terms whose
// first atom is in its block: their atoms lie in its block or in the first
// three atoms of the next block (B >= 3), so the lane adds forces to its own
// atoms in registers and only the next block's first atoms go through shared
// memory, each written by one lane only.  Any other topology uses colour
// classes of atom-disjoint terms, lanes striding over each class.
//
// Atoms beyond N (padding up to L*B) get zero parameters, infinite mass and
// positions 1000 nm away from everything, so they contribute exactly zero.
#pragma once

#include <type_traits>

#include "pamd_device.cuh"
#include "pamd_internal.h"

namespace pamd {

// Launch bounds, chosen by measurement: blocks of up to 256 threads, two per
// SM (128 registers per thread) for up to 3 atoms per lane and one (255)
// above, where the cap would spill; except 5 atoms per lane, whose blocks
// are capped at 128 threads so that three fit per SM at 170 registers (12
// warps instead of 8: 1.7 % faster than the best 256-thread shape on the
// 75-atom chain).  A build may override the block count with
// PAMD_PROP_MIN_BLOCKS.  prop_max_threads (pamd_internal.h) is the host's copy
// of the block-size cap.
template <int B>
struct PropCfg {
    static constexpr int BS = (B % 2 == 1) ? B : B + 1;  // odd stride: conflict-free LDS.128
    static constexpr int MAX_THREADS = prop_max_threads(B);
#ifdef PAMD_PROP_MIN_BLOCKS
    static constexpr int MIN_BLOCKS = PAMD_PROP_MIN_BLOCKS;
#else
    static constexpr int MIN_BLOCKS = (B <= 3) ? 2 : (B == 5 ? 3 : 1);
#endif
};

// Lennard-Jones + Coulomb for one pair.  d = x_j - x_i.  With
// sig2 = sigma_ij^2, eps = 24 sqrt(eps_i eps_j), e2 = 2 eps (exactly) and
// qq = k_e q_i q_j the force on i is -fs * d and on j +fs * d, with
// fs r^2 = eps (2 (s/r)^12 - (s/r)^6) + qq / r = (s/r)^6 (e2 (s/r)^6 - eps) + qq / r;
// e is 4 eps_ij [(s/r)^12 - (s/r)^6] + k_e q_i q_j / r.
template <bool ENERGY>
__device__ __forceinline__ void pair_lj_coul(float dx, float dy, float dz, float sig2, float eps,
                                             float e2, float qq, float& fs, float& e) {
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float rinv = rsqrtf(r2);
    const float rinv2 = rinv * rinv;
    const float s2 = sig2 * rinv2;
    const float s6 = s2 * s2 * s2;
    const float lj = s6 * fmaf(e2, s6, -eps);
    fs = fmaf(qq, rinv, lj) * rinv2;
    if (ENERGY) e = fmaf((eps * (1.0f / 6.0f)) * s6, s6 - 1.0f, qq * rinv);
}

// One tile: the lane's B atoms (registers) against the B atoms of partner
// block J (shared memory).  The partner atoms are taken one at a time (b outer,
// a inner), so that only one partner position, its parameters and its force
// accumulator are live at once; each partner's force goes back to shared
// memory before the next is loaded.  Per accumulator the summation order is
// that of a full B x B sweep (a inner for the partner, b increasing for the
// lane's own atoms).
//
// With TABLE the pair parameters {sigma_ij^2, eps_ij, qq_ij, 2 eps_ij} come
// from a per-tile table in shared memory (entry (b, a) at tab[(b B + a) L];
// the L lanes of a group read consecutive float4s) instead of being mixed
// from the per-atom parameters: the same values (the table holds exactly the
// FP32 products the mixing computes), five fewer FMA-pipe instructions per
// pair.
template <int B, bool MASKED, bool ENERGY, bool TABLE>
__device__ __forceinline__ void pair_tile(const float (&xi)[B], const float (&yi)[B],
                                          const float (&zi)[B], const float (&hsi)[B],
                                          const float (&sei)[B], const float (&qi)[B],
                                          float (&fxi)[B], float (&fyi)[B], float (&fzi)[B],
                                          const float4* pj_s, const float4* cj_s, float4* fj_s,
                                          const float4* tab, int L, unsigned long long mask,
                                          double& e_acc) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const float4 pj = pj_s[b];
        float4 cj = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (!TABLE) cj = cj_s[b];
        float fxj = 0.0f, fyj = 0.0f, fzj = 0.0f;
#pragma unroll
        for (int a = 0; a < B; ++a) {
            const float dx = pj.x - xi[a];
            const float dy = pj.y - yi[a];
            const float dz = pj.z - zi[a];
            float sig2, eps, e2, qq;
            if (TABLE) {
                const float4 t = tab[(b * B + a) * L];
                sig2 = t.x;
                eps = t.y;
                qq = t.z;
                e2 = t.w;
            } else {
                const float sg = hsi[a] + cj.x;
                sig2 = sg * sg;
                eps = sei[a] * cj.y;
                qq = qi[a] * cj.z;
                e2 = eps + eps;
            }
            float fs, e;
            pair_lj_coul<ENERGY>(dx, dy, dz, sig2, eps, e2, qq, fs, e);
            if (MASKED) {
                const bool skip = (mask >> (a * B + b)) & 1ull;
                fs = skip ? 0.0f : fs;
                if (ENERGY) e = skip ? 0.0f : e;
            }
            fxi[a] = fmaf(-fs, dx, fxi[a]);
            fyi[a] = fmaf(-fs, dy, fyi[a]);
            fzi[a] = fmaf(-fs, dz, fzi[a]);
            fxj = fmaf(fs, dx, fxj);
            fyj = fmaf(fs, dy, fyj);
            fzj = fmaf(fs, dz, fzj);
            if (ENERGY) e_acc += (double)e;
        }
        float4 f = fj_s[b];
        f.x += fxj;
        f.y += fyj;
        f.z += fzj;
        fj_s[b] = f;
    }
}

__device__ __forceinline__ void add_force(float4* frc, int s, float fx, float fy, float fz) {
    float4 f = frc[s];
    f.x += fx;
    f.y += fy;
    f.z += fz;
    frc[s] = f;
}

__device__ __forceinline__ float3 f3sub(float3 a, float3 b) {
    return make_float3(a.x - b.x, a.y - b.y, a.z - b.z);
}
__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) {
    return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z));
}
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 f3scale(float s, float3 a) {
    return make_float3(s * a.x, s * a.y, s * a.z);
}
__device__ __forceinline__ float3 f3axpby(float a, float3 x, float b, float3 y) {
    return make_float3(fmaf(a, x.x, b * y.x), fmaf(a, x.y, b * y.y), fmaf(a, x.z, b * y.z));
}

// ---- bonded term kernels on positions; return forces on each atom ----------

// The bonded terms take every length and inverse length from one reciprocal
// square root (MUFU) per squared length, r = r^2 * (1/r), instead of square
// roots and divisions.

// 1/2 k (r - r0)^2 ; force on atom i (atom j gets the opposite)
template <bool ENERGY>
__device__ __forceinline__ float3 bond_force(float3 pi_, float3 pj_, float r0, float k,
                                             double& e_acc) {
    const float3 d = f3sub(pi_, pj_);
    const float r2 = dot3(d, d);
    const float ri = rsqrtf(r2);
    const float r = r2 * ri;
    const float gk = (r0 == 0.0f) ? k : k * (r - r0) * ri;
    if (ENERGY) e_acc += (double)(0.5f * k * (r - r0) * (r - r0));
    return f3scale(-gk, d);
}

// 1/2 k (theta - theta0)^2 with theta the angle at j
template <bool ENERGY>
__device__ __forceinline__ void angle_force(float3 pi_, float3 pj_, float3 pk_, float t0, float kk,
                                            float3& fi, float3& fj, float3& fk, double& e_acc) {
    const float3 u = f3sub(pi_, pj_);
    const float3 w = f3sub(pk_, pj_);
    const float3 uxw = cross3(u, w);
    const float s2 = dot3(uxw, uxw);
    const float rs = rsqrtf(s2);
    const float s = s2 * rs;
    const float cw = dot3(u, w);
    const float dth = atan2f(s, cw) - t0;
    const float gk = kk * dth;
    const float is = gk * rs;
    const float ru = rsqrtf(dot3(u, u)), rw = rsqrtf(dot3(w, w));
    const float cu = cw * (ru * ru), cv = cw * (rw * rw);
    // F_i = -gk dtheta/du = gk (w - cu u)/s ; F_k = gk (u - cv w)/s
    fi = make_float3(is * (w.x - cu * u.x), is * (w.y - cu * u.y), is * (w.z - cu * u.z));
    fk = make_float3(is * (u.x - cv * w.x), is * (u.y - cv * w.y), is * (u.z - cv * w.z));
    fj = make_float3(-fi.x - fk.x, -fi.y - fk.y, -fi.z - fk.z);
    if (ENERGY) e_acc += (double)(0.5f * kk * dth * dth);
}

// k (1 + cos(n phi - phase)); gradient of phi after Blondel & Karplus (1996)
template <bool ENERGY>
__device__ __forceinline__ void dihedral_force(float3 pi_, float3 pj_, float3 pk_, float3 pl_,
                                               float4 prm, float3& fi, float3& fj, float3& fk,
                                               float3& fl, double& e_acc) {
    const float kd = prm.x, nn = prm.y, cph = prm.z, sph = prm.w;
    const float3 F = f3sub(pi_, pj_);
    const float3 G = f3sub(pj_, pk_);
    const float3 H = f3sub(pl_, pk_);
    const float3 A = cross3(F, G);
    const float3 Bv = cross3(H, G);
    const float AA = dot3(A, A), BB = dot3(Bv, Bv);
    const float GG = dot3(G, G);
    const float rlg = rsqrtf(GG);
    const float lg = GG * rlg;
    const float rA = rsqrtf(AA), rB = rsqrtf(BB);
    const float rA2 = rA * rA, rB2 = rB * rB;
    const float rab = rA * rB;
    const float cphi = dot3(A, Bv) * rab;
    // sin phi = ((B x A) . G) / (|A| |B| |G|), and (B x A) . G = -(F . B) |G|^2
    // because B . G = 0, so sin phi = -(F . B) |G| / (|A| |B|)
    const float sphi = -dot3(F, Bv) * lg * rab;
    // cos(n phi), sin(n phi) for n = 1..6 without a loop (straight-line code,
    // so the terms of a lane interleave): multiple-angle formulas up to 3 phi,
    // then n phi = 3 phi + (n - 3) phi for n > 3
    const int n = (int)nn;
    const float c2 = fmaf(cphi + cphi, cphi, -1.0f), s2 = (sphi + sphi) * cphi;
    const float c3 = fmaf(c2, cphi, -s2 * sphi), s3 = fmaf(s2, cphi, c2 * sphi);
    const int m = (n > 3) ? n - 3 : n;
    const float ca = (m == 1) ? cphi : ((m == 2) ? c2 : c3);
    const float sa = (m == 1) ? sphi : ((m == 2) ? s2 : s3);
    const float cn = (n > 3) ? fmaf(c3, ca, -s3 * sa) : ca;
    const float sn = (n > 3) ? fmaf(s3, ca, c3 * sa) : sa;
    const float dEdphi = -kd * nn * (sn * cph - cn * sph);
    const float ia = lg * rA2, ib = lg * rB2;
    const float pa = dot3(F, G) * rA2 * rlg, pb = dot3(H, G) * rB2 * rlg;
    fi = f3scale(dEdphi * ia, A);
    fl = f3scale(-dEdphi * ib, Bv);
    fj = f3axpby(-dEdphi * (ia + pa), A, dEdphi * pb, Bv);
    fk = f3axpby(dEdphi * pa, A, -dEdphi * (pb - ib), Bv);
    if (ENERGY) e_acc += (double)(kd * (1.0f + cn * cph + sn * sph));
}

// scaled Lennard-Jones + Coulomb of a 1-4 pair; force on i
template <bool ENERGY>
__device__ __forceinline__ float3 pair14_force(float3 pi_, float3 pj_, float4 ci, float4 cj,
                                               float s_lj, float s_c, double& e_acc) {
    const float3 d = f3sub(pj_, pi_);
    const float r2 = dot3(d, d);
    const float rinv = rsqrtf(r2);
    const float rinv2 = rinv * rinv;
    const float sig = ci.x + cj.x;
    const float s2 = sig * sig * rinv2;
    const float s6 = s2 * s2 * s2;
    const float eps = ci.y * cj.y;
    const float cq = s_c * ci.z * cj.z * rinv;
    const float lj = s_lj * eps * s6 * fmaf(2.0f, s6, -1.0f);
    const float fs = (lj + cq) * rinv2;
    if (ENERGY) e_acc += (double)(s_lj * (eps * (1.0f / 6.0f)) * s6 * (s6 - 1.0f) + cq);
    return f3scale(-fs, d);
}

// Generic bonded pass: colour by colour, lanes of the group stride over the
// terms of a colour (atom-disjoint, so plain read-modify-writes suffice).
template <bool ENERGY>
__device__ __forceinline__ void bonded_colored(const unsigned char* sm, const TopoLayout& lay,
                                               const float4* prm, const float4* pos, float4* frc,
                                               int L, int g, unsigned gmask, double& e_acc) {
    const int* colors = reinterpret_cast<const int*>(sm + lay.off_colors);
    {
        const BondRec* rec = reinterpret_cast<const BondRec*>(sm + lay.off_bonds);
        const int* cs = colors + 0 * (kMaxColors + 1);
        for (int c = 0; c < lay.n_colors[0]; ++c) {
            for (int t = cs[c] + g; t < cs[c + 1]; t += L) {
                const BondRec b = rec[t];
                const float3 f = bond_force<ENERGY>(f3(pos[b.i]), f3(pos[b.j]), b.r0, b.k, e_acc);
                add_force(frc, b.i, f.x, f.y, f.z);
                add_force(frc, b.j, -f.x, -f.y, -f.z);
            }
            __syncwarp(gmask);
        }
    }
    {
        const AngleRec* rec = reinterpret_cast<const AngleRec*>(sm + lay.off_angles);
        const int* cs = colors + 1 * (kMaxColors + 1);
        for (int c = 0; c < lay.n_colors[1]; ++c) {
            for (int t = cs[c] + g; t < cs[c + 1]; t += L) {
                const AngleRec a = rec[t];
                float3 fi, fj, fk;
                angle_force<ENERGY>(f3(pos[a.i]), f3(pos[a.j]), f3(pos[a.k]), a.t0, a.kk, fi, fj,
                                    fk, e_acc);
                add_force(frc, a.i, fi.x, fi.y, fi.z);
                add_force(frc, a.j, fj.x, fj.y, fj.z);
                add_force(frc, a.k, fk.x, fk.y, fk.z);
            }
            __syncwarp(gmask);
        }
    }
    {
        const DihRec* rec = reinterpret_cast<const DihRec*>(sm + lay.off_dihs);
        const int* cs = colors + 2 * (kMaxColors + 1);
        for (int c = 0; c < lay.n_colors[2]; ++c) {
            for (int t = cs[c] + g; t < cs[c + 1]; t += L) {
                const DihRec h = rec[t];
                float3 fi, fj, fk, fl;
                dihedral_force<ENERGY>(f3(pos[h.i]), f3(pos[h.j]), f3(pos[h.k]), f3(pos[h.l]),
                                       make_float4(h.kd, h.n, h.cos_ph, h.sin_ph), fi, fj, fk, fl,
                                       e_acc);
                add_force(frc, h.i, fi.x, fi.y, fi.z);
                add_force(frc, h.j, fj.x, fj.y, fj.z);
                add_force(frc, h.k, fk.x, fk.y, fk.z);
                add_force(frc, h.l, fl.x, fl.y, fl.z);
            }
            __syncwarp(gmask);
        }
    }
    {
        const Pair14Rec* rec = reinterpret_cast<const Pair14Rec*>(sm + lay.off_p14);
        const int* cs = colors + 3 * (kMaxColors + 1);
        for (int c = 0; c < lay.n_colors[3]; ++c) {
            for (int t = cs[c] + g; t < cs[c + 1]; t += L) {
                const Pair14Rec q = rec[t];
                const float3 f = pair14_force<ENERGY>(f3(pos[q.i]), f3(pos[q.j]), prm[q.i], prm[q.j],
                                                      q.s_lj, q.s_c, e_acc);
                add_force(frc, q.i, f.x, f.y, f.z);
                add_force(frc, q.j, -f.x, -f.y, -f.z);
            }
            __syncwarp(gmask);
        }
    }
}

// Chain bonded pass (B >= 3): the lane's terms start in its block; atom
// offsets o = 0..B+2 relative to the block start, o >= B in the next block.
template <int B, bool ENERGY>
__device__ __forceinline__ void bonded_chain(const unsigned char* sm, const TopoLayout& lay,
                                             const float4* prm, const float4* pos, float4* frc,
                                             int L, int g, const float (&xi)[B],
                                             const float (&yi)[B], const float (&zi)[B],
                                             float (&fx)[B], float (&fy)[B], float (&fz)[B],
                                             double& e_acc) {
    static_assert(B >= 3, "chain pass needs three atoms per lane");
    using C = PropCfg<B>;
    const int i0 = g * B;
    const int N = lay.n_atoms;
    if (i0 + 1 >= N) return;  // no term starts here
    const bool has_next = (g + 1 < L);
    const int nbase = (g + 1) * C::BS;
    float3 sp[3];
    float3 sf[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        sp[m] = has_next ? f3(pos[nbase + m]) : make_float3(0.f, 0.f, 0.f);
        sf[m] = make_float3(0.f, 0.f, 0.f);
    }
    auto P = [&](int o) -> float3 {
        return (o < B) ? make_float3(xi[o < B ? o : 0], yi[o < B ? o : 0], zi[o < B ? o : 0])
                       : sp[o >= B ? o - B : 0];
    };
    auto F = [&](int o, float3 f) {
        if (o < B) {
            fx[o < B ? o : 0] += f.x;
            fy[o < B ? o : 0] += f.y;
            fz[o < B ? o : 0] += f.z;
        } else {
            float3& s = sf[o >= B ? o - B : 0];
            s.x += f.x;
            s.y += f.y;
            s.z += f.z;
        }
    };
    const float2* cb = reinterpret_cast<const float2*>(sm + lay.off_cbond);
    const float2* ca = reinterpret_cast<const float2*>(sm + lay.off_cangle);
    const float4* cd = reinterpret_cast<const float4*>(sm + lay.off_cdih);
#pragma unroll
    for (int a = 0; a < B; ++a) {
        const int d = i0 + a;
        if (d + 1 < N) {  // bond (d, d+1)
            const float2 q = cb[d];
            const float3 f = bond_force<ENERGY>(P(a), P(a + 1), q.x, q.y, e_acc);
            F(a, f);
            F(a + 1, make_float3(-f.x, -f.y, -f.z));
        }
        if (d + 2 < N) {  // angle (d, d+1, d+2)
            const float2 q = ca[d];
            float3 fi, fj, fk;
            angle_force<ENERGY>(P(a), P(a + 1), P(a + 2), q.x, q.y, fi, fj, fk, e_acc);
            F(a, fi);
            F(a + 1, fj);
            F(a + 2, fk);
        }
        if (d + 3 < N) {  // dihedral (d..d+3) and 1-4 pair (d, d+3)
            float3 fi, fj, fk, fl;
            dihedral_force<ENERGY>(P(a), P(a + 1), P(a + 2), P(a + 3), cd[d], fi, fj, fk, fl,
                                   e_acc);
            F(a, fi);
            F(a + 1, fj);
            F(a + 2, fk);
            F(a + 3, fl);
            const int s0 = g * C::BS + a;
            const int s3 = (a + 3 < B) ? (s0 + 3) : (nbase + a + 3 - B);
            const float3 f = pair14_force<ENERGY>(P(a), P(a + 3), prm[s0], prm[s3], lay.s14_lj,
                                                  lay.s14_c, e_acc);
            F(a, f);
            F(a + 3, make_float3(-f.x, -f.y, -f.z));
        }
    }
    if (has_next) {
#pragma unroll
        for (int m = 0; m < 3; ++m) add_force(frc, nbase + m, sf[m].x, sf[m].y, sf[m].z);
    }
}

// Bonded energies of a chain lane's terms (no forces written).
template <int B>
__device__ __forceinline__ void bonded_chain_energy(const unsigned char* sm, const TopoLayout& lay,
                                                    const float4* prm, const float4* pos, int L,
                                                    int g, const float (&xi)[B],
                                                    const float (&yi)[B], const float (&zi)[B],
                                                    double& e_acc) {
    using C = PropCfg<B>;
    const int i0 = g * B;
    const int N = lay.n_atoms;
    const int nbase = (g + 1) * C::BS;
    const bool has_next = (g + 1 < L);
    float3 sp[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) sp[m] = has_next ? f3(pos[nbase + m]) : make_float3(0.f, 0.f, 0.f);
    auto P = [&](int o) -> float3 {
        return (o < B) ? make_float3(xi[o < B ? o : 0], yi[o < B ? o : 0], zi[o < B ? o : 0])
                       : sp[o >= B ? o - B : 0];
    };
    const float2* cb = reinterpret_cast<const float2*>(sm + lay.off_cbond);
    const float2* ca = reinterpret_cast<const float2*>(sm + lay.off_cangle);
    const float4* cd = reinterpret_cast<const float4*>(sm + lay.off_cdih);
#pragma unroll
    for (int a = 0; a < B; ++a) {
        const int d = i0 + a;
        float3 f1, f2, f3_, f4;
        if (d + 1 < N) bond_force<true>(P(a), P(a + 1), cb[d].x, cb[d].y, e_acc);
        if (d + 2 < N) angle_force<true>(P(a), P(a + 1), P(a + 2), ca[d].x, ca[d].y, f1, f2, f3_, e_acc);
        if (d + 3 < N) {
            dihedral_force<true>(P(a), P(a + 1), P(a + 2), P(a + 3), cd[d], f1, f2, f3_, f4, e_acc);
            const int s0 = g * C::BS + a;
            const int s3 = (a + 3 < B) ? (s0 + 3) : (nbase + a + 3 - B);
            pair14_force<true>(P(a), P(a + 3), prm[s0], prm[s3], lay.s14_lj, lay.s14_c, e_acc);
        }
    }
}

// Bonded energies of the generic colour-class layout: lane g takes terms
// g, g+L, ... of every list (no writes, so colours do not matter).
__device__ __forceinline__ void bonded_colored_energy(const unsigned char* sm, const TopoLayout& lay,
                                                      const float4* prm, const float4* pos, int L,
                                                      int g, double& e_acc) {
    float3 f1, f2, f3_, f4;
    const BondRec* br = reinterpret_cast<const BondRec*>(sm + lay.off_bonds);
    for (int t = g; t < lay.n_bonds; t += L)
        bond_force<true>(f3(pos[br[t].i]), f3(pos[br[t].j]), br[t].r0, br[t].k, e_acc);
    const AngleRec* ar = reinterpret_cast<const AngleRec*>(sm + lay.off_angles);
    for (int t = g; t < lay.n_angles; t += L)
        angle_force<true>(f3(pos[ar[t].i]), f3(pos[ar[t].j]), f3(pos[ar[t].k]), ar[t].t0, ar[t].kk,
                          f1, f2, f3_, e_acc);
    const DihRec* dr = reinterpret_cast<const DihRec*>(sm + lay.off_dihs);
    for (int t = g; t < lay.n_dihs; t += L)
        dihedral_force<true>(f3(pos[dr[t].i]), f3(pos[dr[t].j]), f3(pos[dr[t].k]), f3(pos[dr[t].l]),
                             make_float4(dr[t].kd, dr[t].n, dr[t].cos_ph, dr[t].sin_ph), f1, f2,
                             f3_, f4, e_acc);
    const Pair14Rec* pr = reinterpret_cast<const Pair14Rec*>(sm + lay.off_p14);
    for (int t = g; t < lay.n_p14; t += L)
        pair14_force<true>(f3(pos[pr[t].i]), f3(pos[pr[t].j]), prm[pr[t].i], prm[pr[t].j],
                           pr[t].s_lj, pr[t].s_c, e_acc);
}

// Forces on the lane's B atoms (registers fx, fy, fz); positions must already
// be in shared memory and the lane's force slots zeroed, with a __syncwarp
// after both.
template <int B, bool CHAIN, bool ENERGY, bool TABLE = false>
__device__ __forceinline__ void compute_forces(const unsigned char* sm, const TopoLayout& lay,
                                               const float4* prm, const float4* pos, float4* frc,
                                               const unsigned long long* masks, int L, int g,
                                               unsigned gmask, const float (&xi)[B],
                                               const float (&yi)[B], const float (&zi)[B],
                                               const float (&hsi)[B], const float (&sei)[B],
                                               const float (&qi)[B], float (&fx)[B],
                                               float (&fy)[B], float (&fz)[B], double& e_acc) {
    using C = PropCfg<B>;
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
                const float sg = hsi[a] + hsi[b];
                const float eps = sei[a] * sei[b];
                float fs, e;
                pair_lj_coul<ENERGY>(dx, dy, dz, sg * sg, eps, eps + eps, qi[a] * qi[b], fs, e);
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
    // half ring over partner blocks.  Without masked pairs beyond the first
    // ring step (lay.far_masks == 0: a chain with at least 3 atoms per lane)
    // the tiles t >= 2 run the plain code with no test of the mask; otherwise
    // each lane picks the plain or the masked code by its tile's mask.
    const int TH = L / 2;
    auto tile = [&](int t, auto mode) {
        constexpr int MODE = decltype(mode)::value;  // 0 plain, 1 masked, 2 by mask
        const bool active = !(2 * t == L && g >= t);
        if (active) {
            int J = g + t;
            J = (J >= L) ? J - L : J;
            const int sJ = J * C::BS;
            const float4* tab = nullptr;
            if (TABLE)
                tab = reinterpret_cast<const float4*>(sm + lay.off_ptab) + (size_t)(t - 1) * B * B * L + g;
            const unsigned long long m = MODE == 0 ? 0ull : masks[t * L + g];
            if (MODE == 0 || (MODE == 2 && m == 0ull))
                pair_tile<B, false, ENERGY, TABLE>(xi, yi, zi, hsi, sei, qi, fx, fy, fz, pos + sJ,
                                                   prm + sJ, frc + sJ, tab, L, m, e_acc);
            else
                pair_tile<B, true, ENERGY, TABLE>(xi, yi, zi, hsi, sei, qi, fx, fy, fz, pos + sJ,
                                                  prm + sJ, frc + sJ, tab, L, m, e_acc);
        }
        __syncwarp(gmask);
    };
    if (!lay.far_masks) {
        if (TH >= 1) tile(1, std::integral_constant<int, 2>{});
#pragma unroll 1
        for (int t = 2; t <= TH; ++t) tile(t, std::integral_constant<int, 0>{});
    } else {
#pragma unroll 1
        for (int t = 1; t <= TH; ++t) tile(t, std::integral_constant<int, 2>{});
    }
    if constexpr (CHAIN)
        bonded_chain<B, ENERGY>(sm, lay, prm, pos, frc, L, g, xi, yi, zi, fx, fy, fz, e_acc);
    else
        bonded_colored<ENERGY>(sm, lay, prm, pos, frc, L, g, gmask, e_acc);
    __syncwarp(gmask);
#pragma unroll
    for (int a = 0; a < B; ++a) {
        const float4 f = frc[g * C::BS + a];
        fx[a] += f.x;
        fy[a] += f.y;
        fz[a] += f.z;
    }
}

// Potential energy of the lane's share of the replica (FP32 terms summed in
// FP64): its own block's pairs, its half-ring tiles and its bonded terms.
// Reads positions only, so no synchronisation is needed beyond the one that
// published them.
template <int B, bool CHAIN>
__device__ __noinline__ double energy_pass(const unsigned char* sm, const TopoLayout& lay,
                                           const float4* prm, const float4* pos,
                                           const unsigned long long* masks, int L, int g) {
    using C = PropCfg<B>;
    double e_acc = 0.0;
    float xi[B], yi[B], zi[B], hsi[B], sei[B], qi[B];
#pragma unroll
    for (int a = 0; a < B; ++a) {
        const float4 p4 = pos[g * C::BS + a];
        const float4 c4 = prm[g * C::BS + a];
        xi[a] = p4.x; yi[a] = p4.y; zi[a] = p4.z;
        hsi[a] = c4.x; sei[a] = c4.y; qi[a] = c4.z;
    }
    {
        const unsigned long long m = masks[g];
#pragma unroll
        for (int a = 0; a < B; ++a) {
#pragma unroll
            for (int b = a + 1; b < B; ++b) {
                if ((m >> (a * B + b)) & 1ull) continue;
                const float sg = hsi[a] + hsi[b];
                const float eps = sei[a] * sei[b];
                float fs, e;
                pair_lj_coul<true>(xi[b] - xi[a], yi[b] - yi[a], zi[b] - zi[a], sg * sg, eps, eps + eps,
                                   qi[a] * qi[b], fs, e);
                e_acc += (double)e;
            }
        }
    }
    const int TH = L / 2;
    for (int t = 1; t <= TH; ++t) {
        if (2 * t == L && g >= t) continue;
        int J = g + t;
        J = (J >= L) ? J - L : J;
        const unsigned long long m = masks[t * L + g];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const float4 pj = pos[J * C::BS + b];
            const float4 cj = prm[J * C::BS + b];
#pragma unroll
            for (int a = 0; a < B; ++a) {
                if ((m >> (a * B + b)) & 1ull) continue;
                const float sg = hsi[a] + cj.x;
                const float eps = sei[a] * cj.y;
                float fs, e;
                pair_lj_coul<true>(pj.x - xi[a], pj.y - yi[a], pj.z - zi[a], sg * sg, eps, eps + eps,
                                   qi[a] * cj.z, fs, e);
                e_acc += (double)e;
            }
        }
    }
    // bonded terms: reuse the force routines (their force outputs are unused)
    if constexpr (CHAIN) {
        float fx[B], fy[B], fz[B];
        bonded_chain_energy<B>(sm, lay, prm, pos, L, g, xi, yi, zi, e_acc);
        (void)fx; (void)fy; (void)fz;
    } else {
        bonded_colored_energy(sm, lay, prm, pos, L, g, e_acc);
    }
    return e_acc;
}

// Sum over the L lanes of a group (any L), result in every lane.
__device__ __forceinline__ double group_sum(double v, unsigned gmask, int base, int L) {
    double s = 0.0;
    for (int q = 0; q < L; ++q) s += __shfl_sync(gmask, v, base + q);
    return s;
}

// theta BAOAB steps of replica k by the L lanes of one group (lane g of the
// group, lanes base .. base+L-1 of the warp, mask gmask); pos / frc are the
// group's shared-memory slots.  Used by the single-molecule kernel and by the
// batched kernel.
template <int B, bool CHAIN, bool TABLE = false>
__device__ __forceinline__ void advance_replica(const PropParams& p, const unsigned char* sm,
                                                const float4* prm,
                                                const unsigned long long* masks, float4* pos,
                                                float4* frc, long long k, int L, int g, int base,
                                                unsigned gmask) {
    using C = PropCfg<B>;
    const TopoLayout& lay = p.lay;
    const int N = lay.n_atoms, Np = lay.n_pad;
    const uint32_t step_base = (p.dev_counters ? p.dev_counters[0] : 0u) + p.step0;
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
    // s = -1 evaluates the forces of the incoming state; s >= 0 are BAOAB steps
    for (int s = -1; s < p.theta; ++s) {
        if (s >= 0) {
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
                {  // O (padding atoms: zero noise scale, velocity stays 0)
                    const float3 z = normal3_fast(p.seed, (uint32_t)i, (uint32_t)k, step, p.purpose_mol);
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
        }
        compute_forces<B, CHAIN, false, TABLE>(sm, lay, prm, pos, frc, masks, L, g, gmask, xi, yi,
                                               zi, hsi, sei, qi, fx, fy, fz, e_acc);
        if (s >= 0) {
#pragma unroll
            for (int a = 0; a < B; ++a) {                   // B
                vx[a] = fmaf(p.hdt * im[a], fx[a], vx[a]);
                vy[a] = fmaf(p.hdt * im[a], fy[a], vy[a]);
                vz[a] = fmaf(p.hdt * im[a], fz[a], vz[a]);
            }
        }
    }
    // positions in shared memory are those of the last step
    e_acc = energy_pass<B, CHAIN>(sm, lay, prm, pos, masks, L, g);

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
    const double E = group_sum(e_acc, gmask, base, L);
    ek = group_sum(ek, gmask, base, L);
    cx = group_sum(cx, gmask, base, L) / N;
    cy = group_sum(cy, gmask, base, L) / N;
    cz = group_sum(cz, gmask, base, L) / N;
    double r2 = 0.0;
#pragma unroll
    for (int a = 0; a < B; ++a) {
        const int i = g * B + a;
        if (i < N) {
            const double dx = xi[a] - cx, dy = yi[a] - cy, dz = zi[a] - cz;
            r2 += dx * dx + dy * dy + dz * dz;
        }
    }
    r2 = group_sum(r2, gmask, base, L);
    if (g == 0) {
        p.E[k] = E;
        p.ke[k] = ek;
        p.rg[k] = sqrt(r2 / N);
        if (!isfinite(E) && atomicCAS(&p.status[0], 0, PAMD_ENONFINITE) == 0)
            p.status[1] = (int)k;
    }
    __syncwarp(gmask);
}

template <int B, bool CHAIN, bool TABLE>
__global__ void __launch_bounds__(PropCfg<B>::MAX_THREADS, PropCfg<B>::MIN_BLOCKS) propagate_kernel(const PropParams p) {
    using C = PropCfg<B>;
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

    const int L = lay.lanes;
    const int G = 32 / L;
    const int lane = threadIdx.x & 31;
    const int grp = lane / L;
    if (grp >= G) return;  // idle lanes when L does not divide 32
    const int g = lane - grp * L;
    const int base = grp * L;
    const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << base);
    const int slot_local = (threadIdx.x >> 5) * G + grp;
    const int rpb = (blockDim.x >> 5) * G;
    const int slot_f4 = 2 * lay.nk + 1;
    float4* pos = slots + slot_local * slot_f4;
    float4* frc = pos + lay.nk;

    const long long R = p.live ? (long long)*p.live : p.R;
    for (long long k = (long long)blockIdx.x * rpb + slot_local; k < R;
         k += (long long)gridDim.x * rpb)
        advance_replica<B, CHAIN, TABLE>(p, sm, prm, masks, pos, frc, k, L, g, base, gmask);
}

template <int B, bool CHAIN, bool TABLE>
cudaError_t propagate_launch_one(const PropParams* p, int warps, int grid, size_t smem,
                                 cudaStream_t s, int* blocks_per_sm) {
    auto kern = propagate_kernel<B, CHAIN, TABLE>;
    const cudaError_t e = ensure_dyn_smem((const void*)kern, smem);
    if (e != cudaSuccess) return e;
    if (!p) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, warps * 32, smem);
    kern<<<grid, warps * 32, smem, s>>>(*p);
    return cudaGetLastError();
}

// chain: the linear-chain bonded layout; table: the layout carries the
// pair-parameter table (chain layouts only)
template <int B>
cudaError_t propagate_dispatch_b(const PropParams* p, bool chain, bool table, int warps, int grid,
                                 size_t smem, cudaStream_t s, int* blocks_per_sm) {
    if constexpr (B >= 3) {
        if (chain && table) return propagate_launch_one<B, true, true>(p, warps, grid, smem, s, blocks_per_sm);
        if (chain) return propagate_launch_one<B, true, false>(p, warps, grid, smem, s, blocks_per_sm);
    }
    return propagate_launch_one<B, false, false>(p, warps, grid, smem, s, blocks_per_sm);
}

}  // namespace pamd
