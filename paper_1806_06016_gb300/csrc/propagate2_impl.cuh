// propagate2_impl.cuh -- paired persistent BAOAB kernel: each lane group
// advances two replicas at once with packed FP32x2 arithmetic.
//
// Same mapping as propagate_impl.cuh (a group of L lanes per replica, lane g
// owns atoms [g*B, g*B+B), half ring of lane blocks for the nonbonded pairs,
// chain or colour-class bonded pass), but every per-atom quantity is a float2
// holding replica A in .x and replica B in .y.  Both replicas share the
// molecule's parameters and exclusion masks, so one packed instruction
// (__fadd2_rn / __fmul2_rn / __ffma2_rn) does the same step of a pair
// interaction for both replicas, about halving the instructions issued per
// pair.
//
// Sign conventions (chosen so that no packed negation is needed):
//   * the lane keeps its own positions negated (xn = -x); shared memory
//     holds true positions, so d = x_j - x_i = x_j + xn_i is one addition;
//   * the lane accumulates the energy gradient of its own atoms (g = -F =
//     fs * d), while forces on partner atoms (+fs * d) go to shared memory;
//     the total force on an own atom is F = frc - g.
// If R is odd the last group runs its replica twice and writes it once.
#pragma once

#include "propagate_impl.cuh"

namespace pamd {

template <int B>
struct PropCfg2 {
    static constexpr int BS = (B % 2 == 1) ? B : B + 1;
    static constexpr int MIN_BLOCKS = 1;
};

__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Shared-memory slot of one replica pair: positions (x, y of both replicas in
// a float4, z in a float2) and force accumulators in the same layout.
struct Slot2 {
    float4* pxy;  // [nk] (xA, xB, yA, yB)
    float4* fxy;  // [nk]
    float2* pz;   // [nk] (zA, zB)
    float2* fz;   // [nk]
};

__device__ __forceinline__ Slot2 slot2_at(float4* base, int nk) {
    Slot2 s;
    s.pxy = base;
    s.fxy = base + nk;
    s.pz = reinterpret_cast<float2*>(base + 2 * nk);
    s.fz = s.pz + nk;
    return s;
}

// float4s per replica-pair slot: 2 nk float4 + 2 nk float2, plus one of padding
__host__ __device__ inline int slot2_f4(int nk) { return 3 * nk + 1; }

__device__ __forceinline__ float3 pos_of(const Slot2& s, int i, int r) {
    const float4 a = s.pxy[i];
    const float2 z = s.pz[i];
    return r ? make_float3(a.y, a.w, z.y) : make_float3(a.x, a.z, z.x);
}

__device__ __forceinline__ void add_force2(const Slot2& s, int i, float2 fx, float2 fy, float2 fz) {
    float4 a = s.fxy[i];
    float2 z = s.fz[i];
    a.x += fx.x; a.y += fx.y; a.z += fy.x; a.w += fy.y;
    z.x += fz.x; z.y += fz.y;
    s.fxy[i] = a;
    s.fz[i] = z;
}

__device__ __forceinline__ void add_force_r(const Slot2& s, int i, int r, float3 f) {
    float4 a = s.fxy[i];
    float2 z = s.fz[i];
    if (r) { a.y += f.x; a.w += f.y; z.y += f.z; }
    else { a.x += f.x; a.z += f.y; z.x += f.z; }
    s.fxy[i] = a;
    s.fz[i] = z;
}

// Lennard-Jones + Coulomb of pair (i, j) for both replicas; adds fs*d to the
// gradient accumulator of i and to the force accumulator of j.
template <bool MASKED>
__device__ __forceinline__ void pair2(float2 xj, float2 yj, float2 zj, float2 xni, float2 yni,
                                      float2 zni, float sig, float eps, float qq, bool skip,
                                      float2& gxi, float2& gyi, float2& gzi, float2& fxj,
                                      float2& fyj, float2& fzj) {
    const float2 dx = add2(xj, xni);
    const float2 dy = add2(yj, yni);
    const float2 dz = add2(zj, zni);
    const float2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
    const float2 rinv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    const float2 rinv2 = mul2(rinv, rinv);
    const float2 s2 = mul2(bc2(sig * sig), rinv2);
    const float2 s6 = mul2(mul2(s2, s2), s2);
    const float2 lj = mul2(s6, fma2(bc2(eps + eps), s6, bc2(-eps)));  // eps (2 s^12 - s^6)
    float2 fs = mul2(fma2(bc2(qq), rinv, lj), rinv2);
    if (MASKED) fs = skip ? make_float2(0.0f, 0.0f) : fs;
    gxi = fma2(fs, dx, gxi);
    gyi = fma2(fs, dy, gyi);
    gzi = fma2(fs, dz, gzi);
    fxj = fma2(fs, dx, fxj);
    fyj = fma2(fs, dy, fyj);
    fzj = fma2(fs, dz, fzj);
}

// Chain bonded pass for one replica r (B >= 3): terms starting in the lane's
// block; own atoms' forces go into the gradient accumulators (g -= F), the
// next block's first three atoms into shared memory.
template <int B>
__device__ __forceinline__ void bonded_chain2(const unsigned char* sm, const TopoLayout& lay,
                                              const float4* prm, const Slot2& sl, int L, int g,
                                              int r, const float2 (&xn)[B], const float2 (&yn)[B],
                                              const float2 (&zn)[B], float2 (&gx)[B],
                                              float2 (&gy)[B], float2 (&gz)[B]) {
    using C = PropCfg2<B>;
    const int i0 = g * B;
    const int N = lay.n_atoms;
    if (i0 + 1 >= N) return;
    const bool has_next = (g + 1 < L);
    const int nbase = (g + 1) * C::BS;
    float3 sp[3], sf[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        sp[m] = has_next ? pos_of(sl, nbase + m, r) : make_float3(0.f, 0.f, 0.f);
        sf[m] = make_float3(0.f, 0.f, 0.f);
    }
    auto P = [&](int o) -> float3 {
        const int q = o < B ? o : 0;
        return (o < B) ? (r ? make_float3(-xn[q].y, -yn[q].y, -zn[q].y)
                            : make_float3(-xn[q].x, -yn[q].x, -zn[q].x))
                       : sp[o >= B ? o - B : 0];
    };
    auto F = [&](int o, float3 f) {
        if (o < B) {
            const int q = o < B ? o : 0;
            if (r) { gx[q].y -= f.x; gy[q].y -= f.y; gz[q].y -= f.z; }
            else { gx[q].x -= f.x; gy[q].x -= f.y; gz[q].x -= f.z; }
        } else {
            float3& s = sf[o >= B ? o - B : 0];
            s.x += f.x; s.y += f.y; s.z += f.z;
        }
    };
    const float2* cb = reinterpret_cast<const float2*>(sm + lay.off_cbond);
    const float2* ca = reinterpret_cast<const float2*>(sm + lay.off_cangle);
    const float4* cd = reinterpret_cast<const float4*>(sm + lay.off_cdih);
    double e_unused = 0.0;
#pragma unroll
    for (int a = 0; a < B; ++a) {
        const int d = i0 + a;
        if (d + 1 < N) {
            const float2 q = cb[d];
            const float3 f = bond_force<false>(P(a), P(a + 1), q.x, q.y, e_unused);
            F(a, f);
            F(a + 1, make_float3(-f.x, -f.y, -f.z));
        }
        if (d + 2 < N) {
            const float2 q = ca[d];
            float3 fi, fj, fk;
            angle_force<false>(P(a), P(a + 1), P(a + 2), q.x, q.y, fi, fj, fk, e_unused);
            F(a, fi);
            F(a + 1, fj);
            F(a + 2, fk);
        }
        if (d + 3 < N) {
            float3 fi, fj, fk, fl;
            dihedral_force<false>(P(a), P(a + 1), P(a + 2), P(a + 3), cd[d], fi, fj, fk, fl,
                                  e_unused);
            F(a, fi);
            F(a + 1, fj);
            F(a + 2, fk);
            F(a + 3, fl);
            const int s0 = g * C::BS + a;
            const int s3 = (a + 3 < B) ? (s0 + 3) : (nbase + a + 3 - B);
            const float3 f = pair14_force<false>(P(a), P(a + 3), prm[s0], prm[s3], lay.s14_lj,
                                                 lay.s14_c, e_unused);
            F(a, f);
            F(a + 3, make_float3(-f.x, -f.y, -f.z));
        }
    }
    if (has_next) {
#pragma unroll
        for (int m = 0; m < 3; ++m) add_force_r(sl, nbase + m, r, sf[m]);
    }
}

// Generic bonded pass for one replica r: colour classes, forces through
// shared memory (positions from shared memory).
__device__ __forceinline__ void bonded_colored2(const unsigned char* sm, const TopoLayout& lay,
                                                const float4* prm, const Slot2& sl, int L, int g,
                                                int r, unsigned gmask) {
    const int* colors = reinterpret_cast<const int*>(sm + lay.off_colors);
    double e_unused = 0.0;
    {
        const BondRec* rec = reinterpret_cast<const BondRec*>(sm + lay.off_bonds);
        const int* cs = colors;
        for (int c = 0; c < lay.n_colors[0]; ++c) {
            for (int t = cs[c] + g; t < cs[c + 1]; t += L) {
                const BondRec b = rec[t];
                const float3 f = bond_force<false>(pos_of(sl, b.i, r), pos_of(sl, b.j, r), b.r0, b.k,
                                                   e_unused);
                add_force_r(sl, b.i, r, f);
                add_force_r(sl, b.j, r, make_float3(-f.x, -f.y, -f.z));
            }
            __syncwarp(gmask);
        }
    }
    {
        const AngleRec* rec = reinterpret_cast<const AngleRec*>(sm + lay.off_angles);
        const int* cs = colors + (kMaxColors + 1);
        for (int c = 0; c < lay.n_colors[1]; ++c) {
            for (int t = cs[c] + g; t < cs[c + 1]; t += L) {
                const AngleRec a = rec[t];
                float3 fi, fj, fk;
                angle_force<false>(pos_of(sl, a.i, r), pos_of(sl, a.j, r), pos_of(sl, a.k, r), a.t0,
                                   a.kk, fi, fj, fk, e_unused);
                add_force_r(sl, a.i, r, fi);
                add_force_r(sl, a.j, r, fj);
                add_force_r(sl, a.k, r, fk);
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
                dihedral_force<false>(pos_of(sl, h.i, r), pos_of(sl, h.j, r), pos_of(sl, h.k, r),
                                      pos_of(sl, h.l, r),
                                      make_float4(h.kd, h.n, h.cos_ph, h.sin_ph), fi, fj, fk, fl,
                                      e_unused);
                add_force_r(sl, h.i, r, fi);
                add_force_r(sl, h.j, r, fj);
                add_force_r(sl, h.k, r, fk);
                add_force_r(sl, h.l, r, fl);
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
                const float3 f = pair14_force<false>(pos_of(sl, q.i, r), pos_of(sl, q.j, r), prm[q.i],
                                                     prm[q.j], q.s_lj, q.s_c, e_unused);
                add_force_r(sl, q.i, r, f);
                add_force_r(sl, q.j, r, make_float3(-f.x, -f.y, -f.z));
            }
            __syncwarp(gmask);
        }
    }
}

// Total forces on the lane's atoms for both replicas (fx = F).  Positions must
// be in shared memory and the lane's force slots zeroed, with a __syncwarp
// after both.
template <int B, bool CHAIN>
__device__ __forceinline__ void compute_forces2(const unsigned char* sm, const TopoLayout& lay,
                                                const float4* prm, const Slot2& sl,
                                                const unsigned long long* masks, int L, int g,
                                                unsigned gmask, const float2 (&xn)[B],
                                                const float2 (&yn)[B], const float2 (&zn)[B],
                                                const float (&hsi)[B], const float (&sei)[B],
                                                const float (&qi)[B], float2 (&fx)[B],
                                                float2 (&fy)[B], float2 (&fz)[B]) {
    using C = PropCfg2<B>;
    float2 gx[B], gy[B], gz[B];
#pragma unroll
    for (int a = 0; a < B; ++a) gx[a] = gy[a] = gz[a] = make_float2(0.f, 0.f);
    // pairs inside the lane's own block, j positions from shared memory
    {
        const unsigned long long m = masks[g];
#pragma unroll
        for (int b = 1; b < B; ++b) {
            const float4 pj = sl.pxy[g * C::BS + b];
            const float2 zj = sl.pz[g * C::BS + b];
            const float2 xj = make_float2(pj.x, pj.y), yj = make_float2(pj.z, pj.w);
            float2 fxj = make_float2(0.f, 0.f), fyj = fxj, fzj = fxj;
#pragma unroll
            for (int a = 0; a < b; ++a) {
                const bool skip = (m >> (a * B + b)) & 1ull;
                pair2<true>(xj, yj, zj, xn[a], yn[a], zn[a], hsi[a] + hsi[b], sei[a] * sei[b],
                            qi[a] * qi[b], skip, gx[a], gy[a], gz[a], fxj, fyj, fzj);
            }
            // force on own atom b: gradient -= force
            gx[b] = fma2(fxj, bc2(-1.0f), gx[b]);
            gy[b] = fma2(fyj, bc2(-1.0f), gy[b]);
            gz[b] = fma2(fzj, bc2(-1.0f), gz[b]);
        }
    }
    const int TH = L / 2;
#pragma unroll 1
    for (int t = 1; t <= TH; ++t) {
        const bool active = !(2 * t == L && g >= t);
        if (active) {
            int J = g + t;
            J = (J >= L) ? J - L : J;
            float2 xj[B], yj[B], zj[B], fxj[B], fyj[B], fzj[B];
            float4 cj[B];
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const float4 p4 = sl.pxy[J * C::BS + b];
                xj[b] = make_float2(p4.x, p4.y);
                yj[b] = make_float2(p4.z, p4.w);
                zj[b] = sl.pz[J * C::BS + b];
                cj[b] = prm[J * C::BS + b];
                fxj[b] = fyj[b] = fzj[b] = make_float2(0.f, 0.f);
            }
            const unsigned long long m = masks[t * L + g];
            if (m == 0ull) {
#pragma unroll
                for (int a = 0; a < B; ++a)
#pragma unroll
                    for (int b = 0; b < B; ++b)
                        pair2<false>(xj[b], yj[b], zj[b], xn[a], yn[a], zn[a], hsi[a] + cj[b].x,
                                     sei[a] * cj[b].y, qi[a] * cj[b].z, false, gx[a], gy[a], gz[a],
                                     fxj[b], fyj[b], fzj[b]);
            } else {
#pragma unroll
                for (int a = 0; a < B; ++a)
#pragma unroll
                    for (int b = 0; b < B; ++b)
                        pair2<true>(xj[b], yj[b], zj[b], xn[a], yn[a], zn[a], hsi[a] + cj[b].x,
                                    sei[a] * cj[b].y, qi[a] * cj[b].z, (m >> (a * B + b)) & 1ull,
                                    gx[a], gy[a], gz[a], fxj[b], fyj[b], fzj[b]);
            }
#pragma unroll
            for (int b = 0; b < B; ++b) add_force2(sl, J * C::BS + b, fxj[b], fyj[b], fzj[b]);
        }
        __syncwarp(gmask);
    }
    if constexpr (CHAIN) {
        bonded_chain2<B>(sm, lay, prm, sl, L, g, 0, xn, yn, zn, gx, gy, gz);
        bonded_chain2<B>(sm, lay, prm, sl, L, g, 1, xn, yn, zn, gx, gy, gz);
    } else {
        bonded_colored2(sm, lay, prm, sl, L, g, 0, gmask);
        bonded_colored2(sm, lay, prm, sl, L, g, 1, gmask);
    }
    __syncwarp(gmask);
#pragma unroll
    for (int a = 0; a < B; ++a) {
        const float4 f4 = sl.fxy[g * C::BS + a];
        const float2 f2 = sl.fz[g * C::BS + a];
        fx[a] = fma2(gx[a], bc2(-1.0f), make_float2(f4.x, f4.y));
        fy[a] = fma2(gy[a], bc2(-1.0f), make_float2(f4.z, f4.w));
        fz[a] = fma2(gz[a], bc2(-1.0f), f2);
    }
}

// Potential energy of replica r (lane's share), from shared-memory positions.
template <int B, bool CHAIN>
__device__ __noinline__ double energy_pass2(const unsigned char* sm, const TopoLayout& lay,
                                            const float4* prm, const Slot2 sl,
                                            const unsigned long long* masks, int L, int g, int r) {
    using C = PropCfg2<B>;
    double e_acc = 0.0;
    float3 pi_[B];
    float hsi[B], sei[B], qi[B];
#pragma unroll
    for (int a = 0; a < B; ++a) {
        pi_[a] = pos_of(sl, g * C::BS + a, r);
        const float4 c4 = prm[g * C::BS + a];
        hsi[a] = c4.x; sei[a] = c4.y; qi[a] = c4.z;
    }
    {
        const unsigned long long m = masks[g];
#pragma unroll
        for (int a = 0; a < B; ++a)
#pragma unroll
            for (int b = a + 1; b < B; ++b) {
                if ((m >> (a * B + b)) & 1ull) continue;
                const float sg = hsi[a] + hsi[b];
                const float eps = sei[a] * sei[b];
                float fs, e;
                pair_lj_coul<true>(pi_[b].x - pi_[a].x, pi_[b].y - pi_[a].y, pi_[b].z - pi_[a].z,
                                   sg * sg, eps, eps + eps, qi[a] * qi[b], fs, e);
                e_acc += (double)e;
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
            const float3 pj = pos_of(sl, J * C::BS + b, r);
            const float4 cj = prm[J * C::BS + b];
#pragma unroll
            for (int a = 0; a < B; ++a) {
                if ((m >> (a * B + b)) & 1ull) continue;
                const float sg = hsi[a] + cj.x;
                const float eps = sei[a] * cj.y;
                float fs, e;
                pair_lj_coul<true>(pj.x - pi_[a].x, pj.y - pi_[a].y, pj.z - pi_[a].z,
                                   sg * sg, eps, eps + eps, qi[a] * cj.z, fs, e);
                e_acc += (double)e;
            }
        }
    }
    // bonded terms: lane g takes terms g, g+L, ... of every list (reads only)
    if constexpr (CHAIN) {
        const int N = lay.n_atoms;
        const float2* cb = reinterpret_cast<const float2*>(sm + lay.off_cbond);
        const float2* ca = reinterpret_cast<const float2*>(sm + lay.off_cangle);
        const float4* cd = reinterpret_cast<const float4*>(sm + lay.off_cdih);
        auto S = [&](int i) { return (i / B) * C::BS + i % B; };
        float3 f1, f2, f3_, f4;
        for (int d = g; d + 1 < N; d += L)
            bond_force<true>(pos_of(sl, S(d), r), pos_of(sl, S(d + 1), r), cb[d].x, cb[d].y, e_acc);
        for (int d = g; d + 2 < N; d += L)
            angle_force<true>(pos_of(sl, S(d), r), pos_of(sl, S(d + 1), r), pos_of(sl, S(d + 2), r),
                              ca[d].x, ca[d].y, f1, f2, f3_, e_acc);
        for (int d = g; d + 3 < N; d += L) {
            dihedral_force<true>(pos_of(sl, S(d), r), pos_of(sl, S(d + 1), r), pos_of(sl, S(d + 2), r),
                                 pos_of(sl, S(d + 3), r), cd[d], f1, f2, f3_, f4, e_acc);
            pair14_force<true>(pos_of(sl, S(d), r), pos_of(sl, S(d + 3), r), prm[S(d)], prm[S(d + 3)],
                               lay.s14_lj, lay.s14_c, e_acc);
        }
    } else {
        float3 f1, f2, f3_, f4;
        const BondRec* br = reinterpret_cast<const BondRec*>(sm + lay.off_bonds);
        for (int t = g; t < lay.n_bonds; t += L)
            bond_force<true>(pos_of(sl, br[t].i, r), pos_of(sl, br[t].j, r), br[t].r0, br[t].k, e_acc);
        const AngleRec* ar = reinterpret_cast<const AngleRec*>(sm + lay.off_angles);
        for (int t = g; t < lay.n_angles; t += L)
            angle_force<true>(pos_of(sl, ar[t].i, r), pos_of(sl, ar[t].j, r), pos_of(sl, ar[t].k, r),
                              ar[t].t0, ar[t].kk, f1, f2, f3_, e_acc);
        const DihRec* dr = reinterpret_cast<const DihRec*>(sm + lay.off_dihs);
        for (int t = g; t < lay.n_dihs; t += L)
            dihedral_force<true>(pos_of(sl, dr[t].i, r), pos_of(sl, dr[t].j, r), pos_of(sl, dr[t].k, r),
                                 pos_of(sl, dr[t].l, r),
                                 make_float4(dr[t].kd, dr[t].n, dr[t].cos_ph, dr[t].sin_ph), f1, f2,
                                 f3_, f4, e_acc);
        const Pair14Rec* pr = reinterpret_cast<const Pair14Rec*>(sm + lay.off_p14);
        for (int t = g; t < lay.n_p14; t += L)
            pair14_force<true>(pos_of(sl, pr[t].i, r), pos_of(sl, pr[t].j, r), prm[pr[t].i],
                               prm[pr[t].j], pr[t].s_lj, pr[t].s_c, e_acc);
    }
    return e_acc;
}

template <int B, bool CHAIN>
__global__ void __launch_bounds__(256, PropCfg2<B>::MIN_BLOCKS) propagate2_kernel(const PropParams p) {
    using C = PropCfg2<B>;
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
    const int ppb = (blockDim.x >> 5) * G;  // replica pairs per block
    const Slot2 sl = slot2_at(slots + slot_local * slot2_f4(lay.nk), lay.nk);

    const int N = lay.n_atoms, Np = lay.n_pad;
    const uint32_t step_base = (p.dev_counters ? p.dev_counters[0] : 0u) + p.step0;
    const long long npairs = (p.R + 1) / 2;
    const float2 nhdt = bc2(-p.hdt);
    const float2 c1 = bc2(p.c1);

    for (long long q = (long long)blockIdx.x * ppb + slot_local; q < npairs;
         q += (long long)gridDim.x * ppb) {
        const long long kA = 2 * q;
        const bool ghost = (kA + 1 >= p.R);
        const long long kB = ghost ? kA : kA + 1;
        const float* sa = p.state_in + (size_t)kA * 6 * Np;
        const float* sb = p.state_in + (size_t)kB * 6 * Np;
        float2 xn[B], yn[B], zn[B], vx[B], vy[B], vz[B];
        float hsi[B], sei[B], qi[B], hdtim[B], sd[B];
#pragma unroll
        for (int a = 0; a < B; ++a) {
            const int i = g * B + a;
            const int s = g * C::BS + a;
            float2 x, y, z;
            if (i < N) {
                x = make_float2(sa[i], sb[i]);
                y = make_float2(sa[Np + i], sb[Np + i]);
                z = make_float2(sa[2 * Np + i], sb[2 * Np + i]);
                vx[a] = make_float2(sa[3 * Np + i], sb[3 * Np + i]);
                vy[a] = make_float2(sa[4 * Np + i], sb[4 * Np + i]);
                vz[a] = make_float2(sa[5 * Np + i], sb[5 * Np + i]);
            } else {
                x = bc2(1000.0f + 4.0f * (float)i);
                y = z = make_float2(0.f, 0.f);
                vx[a] = vy[a] = vz[a] = make_float2(0.f, 0.f);
            }
            xn[a] = make_float2(-x.x, -x.y);
            yn[a] = make_float2(-y.x, -y.y);
            zn[a] = make_float2(-z.x, -z.y);
            const float4 c = prm[s];
            hsi[a] = c.x;
            sei[a] = c.y;
            qi[a] = c.z;
            hdtim[a] = p.hdt * c.w;
            sd[a] = p.c2kT * sqrtf(c.w);
            sl.pxy[s] = make_float4(x.x, x.y, y.x, y.y);
            sl.pz[s] = z;
            sl.fxy[s] = make_float4(0.f, 0.f, 0.f, 0.f);
            sl.fz[s] = make_float2(0.f, 0.f);
        }
        __syncwarp(gmask);
        float2 fx[B], fy[B], fz[B];
        for (int s = -1; s < p.theta; ++s) {
            if (s >= 0) {
                const uint32_t step = step_base + (uint32_t)s;
#pragma unroll
                for (int a = 0; a < B; ++a) {
                    const int i = g * B + a;
                    const float2 h = bc2(hdtim[a]);
                    vx[a] = fma2(h, fx[a], vx[a]);                   // B
                    vy[a] = fma2(h, fy[a], vy[a]);
                    vz[a] = fma2(h, fz[a], vz[a]);
                    xn[a] = fma2(nhdt, vx[a], xn[a]);                // A (xn = -x)
                    yn[a] = fma2(nhdt, vy[a], yn[a]);
                    zn[a] = fma2(nhdt, vz[a], zn[a]);
                    if (i < N) {                                     // O
                        const float3 za = normal3_fast(p.seed, (uint32_t)i, (uint32_t)kA, step, p.purpose_mol);
                        const float3 zb = normal3_fast(p.seed, (uint32_t)i, (uint32_t)kB, step, p.purpose_mol);
                        const float2 sdv = bc2(sd[a]);
                        vx[a] = fma2(c1, vx[a], mul2(sdv, make_float2(za.x, zb.x)));
                        vy[a] = fma2(c1, vy[a], mul2(sdv, make_float2(za.y, zb.y)));
                        vz[a] = fma2(c1, vz[a], mul2(sdv, make_float2(za.z, zb.z)));
                    }
                    xn[a] = fma2(nhdt, vx[a], xn[a]);                // A
                    yn[a] = fma2(nhdt, vy[a], yn[a]);
                    zn[a] = fma2(nhdt, vz[a], zn[a]);
                    const int sl_i = g * C::BS + a;
                    sl.pxy[sl_i] = make_float4(-xn[a].x, -xn[a].y, -yn[a].x, -yn[a].y);
                    sl.pz[sl_i] = make_float2(-zn[a].x, -zn[a].y);
                    sl.fxy[sl_i] = make_float4(0.f, 0.f, 0.f, 0.f);
                    sl.fz[sl_i] = make_float2(0.f, 0.f);
                }
                __syncwarp(gmask);
            }
            compute_forces2<B, CHAIN>(sm, lay, prm, sl, masks, L, g, gmask, xn, yn, zn, hsi, sei,
                                      qi, fx, fy, fz);
            if (s >= 0) {
#pragma unroll
                for (int a = 0; a < B; ++a) {                        // B
                    const float2 h = bc2(hdtim[a]);
                    vx[a] = fma2(h, fx[a], vx[a]);
                    vy[a] = fma2(h, fy[a], vy[a]);
                    vz[a] = fma2(h, fz[a], vz[a]);
                }
            }
        }
        const double EA = energy_pass2<B, CHAIN>(sm, lay, prm, sl, masks, L, g, 0);
        const double EB = energy_pass2<B, CHAIN>(sm, lay, prm, sl, masks, L, g, 1);

        // write back and per-replica observables
        double ek[2] = {0.0, 0.0}, cx[2] = {0, 0}, cy[2] = {0, 0}, cz[2] = {0, 0};
#pragma unroll
        for (int a = 0; a < B; ++a) {
            const int i = g * B + a;
            if (i < N) {
                const double m = (double)p.masses[i];
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const long long k = r ? kB : kA;
                    const float x = r ? -xn[a].y : -xn[a].x;
                    const float y = r ? -yn[a].y : -yn[a].x;
                    const float z = r ? -zn[a].y : -zn[a].x;
                    const float u = r ? vx[a].y : vx[a].x;
                    const float v = r ? vy[a].y : vy[a].x;
                    const float w = r ? vz[a].y : vz[a].x;
                    if (!(r == 1 && ghost)) {
                        float* so = p.state_out + (size_t)k * 6 * Np;
                        if (p.theta > 0) {
                            so[i] = x; so[Np + i] = y; so[2 * Np + i] = z;
                            so[3 * Np + i] = u; so[4 * Np + i] = v; so[5 * Np + i] = w;
                        }
                        if (p.fout) {
                            float* fo = p.fout + (size_t)k * 3 * Np;
                            fo[i] = r ? fx[a].y : fx[a].x;
                            fo[Np + i] = r ? fy[a].y : fy[a].x;
                            fo[2 * Np + i] = r ? fz[a].y : fz[a].x;
                        }
                    }
                    ek[r] += 0.5 * m * ((double)u * u + (double)v * v + (double)w * w);
                    cx[r] += x;
                    cy[r] += y;
                    cz[r] += z;
                }
            }
        }
        double E[2] = {group_sum(EA, gmask, base, L), group_sum(EB, gmask, base, L)};
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            ek[r] = group_sum(ek[r], gmask, base, L);
            cx[r] = group_sum(cx[r], gmask, base, L) / N;
            cy[r] = group_sum(cy[r], gmask, base, L) / N;
            cz[r] = group_sum(cz[r], gmask, base, L) / N;
        }
        double r2[2] = {0.0, 0.0};
#pragma unroll
        for (int a = 0; a < B; ++a) {
            const int i = g * B + a;
            if (i < N) {
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const double dx = (r ? -xn[a].y : -xn[a].x) - cx[r];
                    const double dy = (r ? -yn[a].y : -yn[a].x) - cy[r];
                    const double dz = (r ? -zn[a].y : -zn[a].x) - cz[r];
                    r2[r] += dx * dx + dy * dy + dz * dz;
                }
            }
        }
        r2[0] = group_sum(r2[0], gmask, base, L);
        r2[1] = group_sum(r2[1], gmask, base, L);
        if (g == 0) {
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                if (r == 1 && ghost) break;
                const long long k = r ? kB : kA;
                p.E[k] = E[r];
                p.ke[k] = ek[r];
                p.rg[k] = sqrt(r2[r] / N);
                if (!isfinite(E[r]) && atomicCAS(&p.status[0], 0, PAMD_ENONFINITE) == 0)
                    p.status[1] = (int)k;
            }
        }
        __syncwarp(gmask);
    }
}

template <int B, bool CHAIN>
cudaError_t propagate2_launch_one(const PropParams* p, int warps, int grid, size_t smem,
                                  cudaStream_t s, int* blocks_per_sm) {
    auto kern = propagate2_kernel<B, CHAIN>;
    const cudaError_t e = ensure_dyn_smem((const void*)kern, smem);
    if (e != cudaSuccess) return e;
    if (!p) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, warps * 32, smem);
    kern<<<grid, warps * 32, smem, s>>>(*p);
    return cudaGetLastError();
}

template <int B>
cudaError_t propagate2_dispatch_b(const PropParams* p, bool chain, int warps, int grid,
                                  size_t smem, cudaStream_t s, int* blocks_per_sm) {
    if constexpr (B >= 3) {
        if (chain) return propagate2_launch_one<B, true>(p, warps, grid, smem, s, blocks_per_sm);
    }
    return propagate2_launch_one<B, false>(p, warps, grid, smem, s, blocks_per_sm);
}

}  // namespace pamd
