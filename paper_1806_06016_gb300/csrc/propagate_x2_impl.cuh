// propagate_x2_impl.cuh -- persistent BAOAB Langevin kernel (PAMD scheme,
// step 3) with the nonbonded pair arithmetic in packed FP32x2 instructions.
//
// Same replica mapping as propagate_impl.cuh: a replica is owned by L lanes
// of a warp (G = floor(32/L) replicas per warp), lane g owns the B atoms
// [gB, gB+B), nonbonded pairs follow the half ring of lane blocks (step t:
// block g against block (g+t) mod L).  What differs:
//
// * Packed arithmetic.  The lane's own atoms are held as P = floor(B/2)
//   register pairs (atoms 2p, 2p+1) plus one scalar atom when B is odd.  One
//   partner atom against one own pair is evaluated by add/mul/fma.rn.f32x2
//   instructions (two FP32 results per instruction: the same FP32 roundings
//   as two scalar instructions, half the issue slots).  The reciprocal square
//   root stays scalar (no packed form).
// * Partner atoms are read from shared memory already duplicated and with
//   their coordinates negated, {-x,-x,-y,-y} and {-z,-z,q,q} per atom, so that
//   d = x_own + (-x_partner) is one add and no instruction is spent forming
//   the broadcast operand of a packed instruction; the per-atom mixing
//   parameters {sigma/2, sigma/2, sqrt(24 eps), sqrt(24 eps)} sit in a
//   per-block table.  Own sqrt(24 eps) are kept negated, so -eps_ij is a
//   product as well: the packed path needs no sign changes.
// * Forces on partner atoms are summed in registers over the tile and handed
//   to the owner lane with warp shuffles (lane g receives from lane g - t the
//   forces on its own block), so shared memory holds positions only and the
//   pair loop has no shared-memory stores.
// * Chain bonded terms share their geometry (bond vectors, normals, dot
//   products) between consecutive terms; forces on the next block's first
//   three atoms are also handed over by shuffles.  The scaled 1-4 pairs,
//   which in a chain always fall in the own block or the t = 1 tile, are
//   evaluated there with their scale factors instead of being masked out and
//   recomputed with the bonded terms.
//
// Linear-chain layouts only (B >= 3); other topologies use propagate_impl.cuh.
#pragma once

#include <type_traits>

#include "propagate_impl.cuh"

namespace pamd {

template <int B>
struct X2Cfg {
    static constexpr int P = B / 2;             // packed own-atom pairs
    static constexpr bool TAIL = (B % 2) == 1;  // one scalar own atom
    static constexpr int BS = (B % 2 == 1) ? B : B + 1;
    static constexpr int MAX_THREADS = kPackedMaxThreads;
#ifdef PAMD_X2_MIN_BLOCKS
    static constexpr int MIN_BLOCKS = PAMD_X2_MIN_BLOCKS;
#else
    static constexpr int MIN_BLOCKS = (B <= 4) ? 4 : 3;
#endif
};

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

// A point about 1000 nm or more from the molecule, distinct for every index
// and never collinear with the points of the two neighbouring indices: where
// padding atoms (and the missing next block of the last lane) sit.
__device__ __forceinline__ float3 far_point(int i) {
    return make_float3(1000.0f + 4.0f * (float)i, 2.0f * (float)(i & 1), 2.0f * (float)((i >> 1) & 1));
}

// atan2(y, x) for y >= 0 (a bond angle from |u x w| and u . w), without
// branches: t = min(|x|, y) / max(|x|, y) in [0, 1], atan(t) = t P(t^2) with
// P a degree-7 polynomial fitted to atan(t)/t on [0, 1] (least squares with
// Lawson reweighting toward the minimax fit; largest error 1.3e-7 rad when
// evaluated in FP32), then pi/2 - atan(t) when y > |x| and pi - (...) when
// x < 0.
__device__ __forceinline__ float atan2_nonneg(float y, float x) {
    const float ax = fabsf(x);
    const float mn = fminf(ax, y), mx = fmaxf(ax, y);
    const float t = mn / mx;
    const float t2 = t * t;
    float p = -0.00405456218868494f;
    p = fmaf(p, t2, 0.021862944588065147f);
    p = fmaf(p, t2, -0.0559123195707798f);
    p = fmaf(p, t2, 0.096421979367733f);
    p = fmaf(p, t2, -0.1390863060951233f);
    p = fmaf(p, t2, 0.19946566224098206f);
    p = fmaf(p, t2, -0.33329859375953674f);
    p = fmaf(p, t2, 0.9999993443489075f);
    float a = p * t;
    a = (y > ax) ? 1.57079632679489662f - a : a;
    return (x < 0.0f) ? 3.14159265358979324f - a : a;
}

// Own atoms of a lane: packed pairs plus the scalar tail.
template <int B>
struct Own {
    static constexpr int P = X2Cfg<B>::P;
    float2 x[P > 0 ? P : 1], y[P > 0 ? P : 1], z[P > 0 ? P : 1];
    float xt, yt, zt;
    __device__ __forceinline__ float gx(int a) const {
        return (a < 2 * P) ? ((a & 1) ? x[a >> 1].y : x[a >> 1].x) : xt;
    }
    __device__ __forceinline__ float gy(int a) const {
        return (a < 2 * P) ? ((a & 1) ? y[a >> 1].y : y[a >> 1].x) : yt;
    }
    __device__ __forceinline__ float gz(int a) const {
        return (a < 2 * P) ? ((a & 1) ? z[a >> 1].y : z[a >> 1].x) : zt;
    }
    __device__ __forceinline__ void add(int a, float vx, float vy, float vz) {
        if (a < 2 * P) {
            if (a & 1) {
                x[a >> 1].y += vx;
                y[a >> 1].y += vy;
                z[a >> 1].y += vz;
            } else {
                x[a >> 1].x += vx;
                y[a >> 1].x += vy;
                z[a >> 1].x += vz;
            }
        } else {
            xt += vx;
            yt += vy;
            zt += vz;
        }
    }
    __device__ __forceinline__ void set(int a, float vx, float vy, float vz) {
        if (a < 2 * P) {
            if (a & 1) {
                x[a >> 1].y = vx;
                y[a >> 1].y = vy;
                z[a >> 1].y = vz;
            } else {
                x[a >> 1].x = vx;
                y[a >> 1].x = vy;
                z[a >> 1].x = vz;
            }
        } else {
            xt = vx;
            yt = vy;
            zt = vz;
        }
    }
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int p = 0; p < (P > 0 ? P : 1); ++p) x[p] = y[p] = z[p] = make_float2(0.f, 0.f);
        xt = yt = zt = 0.f;
    }
};

// Masks of the t = 1 tile of a chain with the usual exclusions (bit a*B + b:
// own atom a of block g against atom b of block g + 1, B + b - a apart):
// excluded pairs (at most 2 apart) and scaled 1-4 pairs (3 apart), or with
// only14 the 1-4 pairs alone.
template <int B>
__host__ __device__ constexpr unsigned long long std_t1_mask(bool only14) {
    unsigned long long m = 0ull;
    for (int a = 0; a < B; ++a)
        for (int b = 0; b < B; ++b) {
            const int d = B + b - a;
            if (d == 3 || (!only14 && d <= 2)) m |= 1ull << (a * B + b);
        }
    return m;
}

// Factors of a pair left out of the plain nonbonded sum: (0, 0) when it is
// excluded, (LJ scale, Coulomb scale) when it is a scaled 1-4 pair, else
// (1, 1).  Applied to eps, 2 eps and qq, which the pair force is linear in.
__device__ __forceinline__ float2 pair_factors(unsigned long long mask, unsigned long long m14,
                                               int bit, float s_lj, float s_c) {
    const bool out = (mask >> bit) & 1ull;
    const bool is14 = (m14 >> bit) & 1ull;
    return make_float2(out ? (is14 ? s_lj : 0.0f) : 1.0f, out ? (is14 ? s_c : 0.0f) : 1.0f);
}

// One partner atom (duplicated operands, negated coordinates) against the
// lane's own atoms.  d = x_own - x_partner; the force on an own atom is +fs d,
// on the partner -fs d; the partner's share is summed into (gx, gy, gz) as
// +fs d (the caller subtracts it).  nse holds -sqrt(24 eps) of the own atoms:
// neps = -eps_ij and e2 = -2 neps = 2 eps_ij.  In a masked tile the own/partner
// pair of bit a*B + b takes the factors of pair_factors.
template <int B, bool MASKED>
__device__ __forceinline__ void partner_x2(const Own<B>& r, const Own<B>& hs, const Own<B>& nse,
                                           const Own<B>& qq, Own<B>& f, float4 pa, float4 pb,
                                           float4 pp, int b, unsigned long long mask,
                                           unsigned long long m14, float s_lj, float s_c,
                                           float& gx, float& gy, float& gz) {
    using C = X2Cfg<B>;
    const float2 nxj = f2(pa.x, pa.y), nyj = f2(pa.z, pa.w), nzj = f2(pb.x, pb.y);
    const float2 qj = f2(pb.z, pb.w), hj = f2(pp.x, pp.y), ej = f2(pp.z, pp.w);
    const float2 m2 = f2(-2.0f);
    float2 Gx, Gy, Gz;
#pragma unroll
    for (int p = 0; p < C::P; ++p) {
        const float2 dx = add2(r.x[p], nxj);
        const float2 dy = add2(r.y[p], nyj);
        const float2 dz = add2(r.z[p], nzj);
        const float2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
        const float2 rinv = f2(rsqrtf(r2.x), rsqrtf(r2.y));
        const float2 rinv2 = mul2(rinv, rinv);
        const float2 sg = add2(hs.x[p], hj);
        const float2 s2 = mul2(mul2(sg, sg), rinv2);
        const float2 s6 = mul2(mul2(s2, s2), s2);
        float2 neps = mul2(nse.x[p], ej);
        float2 q2 = mul2(qq.x[p], qj);
        if (MASKED) {
            const float2 k0 = pair_factors(mask, m14, (2 * p) * B + b, s_lj, s_c);
            const float2 k1 = pair_factors(mask, m14, (2 * p + 1) * B + b, s_lj, s_c);
            neps = mul2(neps, f2(k0.x, k1.x));
            q2 = mul2(q2, f2(k0.y, k1.y));
        }
        const float2 e2 = mul2(neps, m2);
        const float2 lj = mul2(s6, fma2(e2, s6, neps));
        const float2 fs = mul2(fma2(q2, rinv, lj), rinv2);
        f.x[p] = fma2(fs, dx, f.x[p]);
        f.y[p] = fma2(fs, dy, f.y[p]);
        f.z[p] = fma2(fs, dz, f.z[p]);
        if (p == 0) {
            Gx = mul2(fs, dx);
            Gy = mul2(fs, dy);
            Gz = mul2(fs, dz);
        } else {
            Gx = fma2(fs, dx, Gx);
            Gy = fma2(fs, dy, Gy);
            Gz = fma2(fs, dz, Gz);
        }
    }
    gx = Gx.x + Gx.y;
    gy = Gy.x + Gy.y;
    gz = Gz.x + Gz.y;
    if (C::TAIL) {
        const float dx = r.xt + pa.x, dy = r.yt + pa.z, dz = r.zt + pb.x;
        const float sg = hs.xt + pp.x;
        float neps = nse.xt * pp.z;
        float qt = qq.xt * pb.z;
        if (MASKED) {
            const float2 k = pair_factors(mask, m14, (B - 1) * B + b, s_lj, s_c);
            neps *= k.x;
            qt *= k.y;
        }
        float fs, e;
        pair_lj_coul<false>(dx, dy, dz, sg * sg, -neps, -2.0f * neps, qt, fs, e);
        // pair_lj_coul's fs multiplies d = x_j - x_i; here d = x_i - x_j
        f.xt = fmaf(fs, dx, f.xt);
        f.yt = fmaf(fs, dy, f.yt);
        f.zt = fmaf(fs, dz, f.zt);
        gx = fmaf(fs, dx, gx);
        gy = fmaf(fs, dy, gy);
        gz = fmaf(fs, dz, gz);
    }
}

// Chain bonded pass (bonds, angles and dihedrals starting in the lane's
// block): forces on the own atoms go to f, those on the next block's first
// three atoms to sf.  Every lane evaluates B terms of each kind without
// branches: the term parameters past the chain's end are zero (the topology
// table has one entry per atom slot), and padding atoms and the missing next
// block of the last lane sit at distinct, non-collinear points far away (so a
// term with zero parameters gives exactly zero, never 0 * inf).
template <int B>
__device__ __forceinline__ void bonded_chain_x2(const unsigned char* sm, const TopoLayout& lay,
                                                const float4* prm, const float4* posA,
                                                const float4* posB, int L, int g, const Own<B>& r,
                                                Own<B>& f, float3 (&sf)[3]) {
    using C = X2Cfg<B>;
    const int i0 = g * B;
    const bool has_next = (g + 1 < L);
    const int nbase = (g + 1) * C::BS;
    float3 sp[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        sf[m] = make_float3(0.f, 0.f, 0.f);
        if (has_next) {  // stored negated
            const float4 a = posA[nbase + m];
            const float4 c = posB[nbase + m];
            sp[m] = make_float3(-a.x, -a.z, -c.x);
        } else {
            sp[m] = far_point(2000 + m);
        }
    }
    auto P = [&](int o) -> float3 {
        return (o < B) ? make_float3(r.gx(o < B ? o : 0), r.gy(o < B ? o : 0), r.gz(o < B ? o : 0))
                       : sp[o >= B ? o - B : 0];
    };
    auto F = [&](int o, float3 v) {
        if (o < B) {
            f.add(o < B ? o : 0, v.x, v.y, v.z);
        } else {
            float3& s = sf[o >= B ? o - B : 0];
            s.x += v.x;
            s.y += v.y;
            s.z += v.z;
        }
    };
    const float2* cb = reinterpret_cast<const float2*>(sm + lay.off_cbond);
    const float2* ca = reinterpret_cast<const float2*>(sm + lay.off_cangle);
    const float4* cd = reinterpret_cast<const float4*>(sm + lay.off_cdih);
    // Geometry shared by consecutive terms: bond vectors b_k = P(k+1) - P(k)
    // with |b_k|^2 and 1/|b_k|, normals c_k = b_k x b_{k+1} with |c_k|^2 and
    // 1/|c_k|, and d_k = b_k . b_{k+1}.  Bond a uses b_a; the angle at a+1
    // uses b_a, b_{a+1}, c_a, d_a; the dihedral (a..a+3) uses A = c_a,
    // B = c_{a+1}, G = -b_{a+1} and d_a, d_{a+1} (the torsion's F.G and H.G).
    float3 bv[B + 2];
    float bb[B + 2], rb[B + 2];
#pragma unroll
    for (int k = 0; k < B + 2; ++k) {
        bv[k] = f3sub(P(k + 1), P(k));
        bb[k] = dot3(bv[k], bv[k]);
        rb[k] = rsqrtf(bb[k]);
    }
    float3 cv[B + 1];
    float cc[B + 1], rc[B + 1], dd[B + 1];
#pragma unroll
    for (int k = 0; k < B + 1; ++k) {
        cv[k] = cross3(bv[k], bv[k + 1]);
        cc[k] = dot3(cv[k], cv[k]);
        rc[k] = rsqrtf(cc[k]);
        dd[k] = dot3(bv[k], bv[k + 1]);
    }
#pragma unroll
    for (int a = 0; a < B; ++a) {
        const int d = i0 + a;
        {  // bond (d, d+1): 1/2 k (r - r0)^2, force on d is +g b_a
            const float2 q = cb[d];
            const float r = bb[a] * rb[a];
            const float gk = (q.x == 0.0f) ? q.y : q.y * (r - q.x) * rb[a];
            const float3 fb = f3scale(gk, bv[a]);
            F(a, fb);
            F(a + 1, make_float3(-fb.x, -fb.y, -fb.z));
        }
        {  // angle (d, d+1, d+2) at d+1: u = -b_a, w = b_{a+1}, |u x w| = |c_a|, u.w = -d_a
            const float2 q = ca[d];
            const float cw = -dd[a];
            const float dth = atan2_nonneg(cc[a] * rc[a], cw) - q.x;
            const float is = q.y * dth * rc[a];
            const float cu = cw * (rb[a] * rb[a]), cvv = cw * (rb[a + 1] * rb[a + 1]);
            // F_i = is (w - cu u), F_k = is (u - cv w), F_j = -F_i - F_k
            const float3 fi = f3scale(is, f3axpby(1.0f, bv[a + 1], cu, bv[a]));
            const float3 fk = f3scale(-is, f3axpby(1.0f, bv[a], cvv, bv[a + 1]));
            F(a, fi);
            F(a + 1, make_float3(-fi.x - fk.x, -fi.y - fk.y, -fi.z - fk.z));
            F(a + 2, fk);
        }
        {  // dihedral (d..d+3), gradient of phi after Blondel & Karplus (1996)
            const float4 prm_d = cd[d];
            const float kd = prm_d.x, nn = prm_d.y, cph = prm_d.z, sph = prm_d.w;
            const float3 A = cv[a], Bn = cv[a + 1];
            const float rlg = rb[a + 1], lg = bb[a + 1] * rlg;
            const float rA2 = rc[a] * rc[a], rB2 = rc[a + 1] * rc[a + 1];
            const float rab = rc[a] * rc[a + 1];
            const float cphi = dot3(A, Bn) * rab;
            // sin phi = -(F . B) |G| / (|A||B|) with F = -b_a
            const float sphi = dot3(bv[a], Bn) * lg * rab;
            const int n = (int)nn;
            const float c2 = fmaf(cphi + cphi, cphi, -1.0f), s2 = (sphi + sphi) * cphi;
            const float c3 = fmaf(c2, cphi, -s2 * sphi), s3 = fmaf(s2, cphi, c2 * sphi);
            const int m = (n > 3) ? n - 3 : n;
            const float cA = (m == 1) ? cphi : ((m == 2) ? c2 : c3);
            const float sA = (m == 1) ? sphi : ((m == 2) ? s2 : s3);
            const float cn = (n > 3) ? fmaf(c3, cA, -s3 * sA) : cA;
            const float sn = (n > 3) ? fmaf(s3, cA, c3 * sA) : sA;
            const float dEdphi = -kd * nn * (sn * cph - cn * sph);
            const float ia = lg * rA2, ib = lg * rB2;
            // F.G = d_a, H.G = -d_{a+1} (F = -b_a, G = -b_{a+1}, H = b_{a+2})
            const float pa = dd[a] * rA2 * rlg, pb = -dd[a + 1] * rB2 * rlg;
            F(a, f3scale(dEdphi * ia, A));
            F(a + 1, f3axpby(-dEdphi * (ia + pa), A, dEdphi * pb, Bn));
            F(a + 2, f3axpby(dEdphi * pa, A, -dEdphi * (pb - ib), Bn));
            F(a + 3, f3scale(-dEdphi * ib, Bn));
        }
    }
}

// Partner-side sums (g) of one partner atom go to the lane that owns it; this
// lane receives from `src` the sums for its own atom b (force = -sum).
template <int B>
__device__ __forceinline__ void hand_over(Own<B>& f, int b, float gx, float gy, float gz,
                                          unsigned gmask, int src) {
    const float rx = __shfl_sync(gmask, gx, src);
    const float ry = __shfl_sync(gmask, gy, src);
    const float rz = __shfl_sync(gmask, gz, src);
    f.add(b, -rx, -ry, -rz);
}

// Forces on the lane's own atoms (f).  Positions must be in shared memory
// (posA/posB of the replica), published by a __syncwarp.  Every lane of the
// group must call this (the hand-over of partner forces is a warp shuffle).
template <int B>
__device__ __forceinline__ void forces_x2(const unsigned char* sm, const TopoLayout& lay,
                                          const float4* prm, const float4* dprm,
                                          const unsigned long long* masks, const float4* posA,
                                          const float4* posB, int L, int g, int base,
                                          unsigned gmask, const Own<B>& r, const Own<B>& hs,
                                          const Own<B>& nse, const Own<B>& qq, Own<B>& f) {
    using C = X2Cfg<B>;
    // 1-4 pairs of a chain lie in the own block or the t = 1 tile: they are
    // evaluated there with their scale factors, not in the bonded pass
    const unsigned long long* m14s = reinterpret_cast<const unsigned long long*>(sm + lay.off_m14);
    const float s_lj = lay.s14_lj, s_c = lay.s14_c;
    f.zero();
    // pairs inside the lane's own block (the 1-2/1-3/1-4 pairs live here).
    // With the usual chain exclusions the pair pattern of a block is the same
    // for every lane: atoms d = b - a apart are excluded for d <= 2 and
    // scaled for d = 3, which the unrolled loop resolves at compile time
    // (padding slots carry zero parameters, so leaving their pairs out by
    // position changes nothing); otherwise the block's masks decide.
    auto own_pair = [&](int a, int b, float kx, float ky) {
        const float dx = r.gx(b) - r.gx(a), dy = r.gy(b) - r.gy(a), dz = r.gz(b) - r.gz(a);
        const float sg = hs.gx(a) + hs.gx(b);
        const float eps = nse.gx(a) * nse.gx(b) * kx;
        float fs, e;
        pair_lj_coul<false>(dx, dy, dz, sg * sg, eps, eps + eps, qq.gx(a) * qq.gx(b) * ky, fs, e);
        f.add(a, -fs * dx, -fs * dy, -fs * dz);
        f.add(b, fs * dx, fs * dy, fs * dz);
    };
    if (lay.std_chain) {
#pragma unroll
        for (int a = 0; a < B; ++a) {
#pragma unroll
            for (int b = a + 3; b < B; ++b) {
                if (b - a == 3)
                    own_pair(a, b, s_lj, s_c);
                else
                    own_pair(a, b, 1.0f, 1.0f);
            }
        }
    } else {
        const unsigned long long m = masks[g], m4 = m14s[g];
#pragma unroll
        for (int a = 0; a < B; ++a) {
#pragma unroll
            for (int b = a + 1; b < B; ++b) {
                const float2 k = pair_factors(m, m4, a * B + b, s_lj, s_c);
                own_pair(a, b, k.x, k.y);
            }
        }
    }
    // half ring over partner blocks: steps 1..(L-1)/2 give every lane a
    // partner block; for even L the antipodal step L/2 follows, where only
    // lanes g < L/2 work.  Lane g receives from lane g - t the forces on its
    // own atom b.  The partner sums of a whole tile are handed over after
    // it, so that the partners' arithmetic can interleave.
    // mode 0: plain code; 1: the tile's masks from the table; 2: the t = 1
    // tile of a chain with the usual exclusions, whose masks are fixed by
    // position (own atom a against partner b, B + b - a apart) except on the
    // last lane, whose t = 1 partner is block 0 and has none
    auto tile = [&](int t, auto mode) {
        constexpr int MODE = decltype(mode)::value;
        constexpr bool MASKED = MODE != 0;
        int J = g + t;
        J = (J >= L) ? J - L : J;
        const int sJ = J * C::BS;
        int src = g - t;
        src = (src < 0) ? src + L : src;
        unsigned long long m = 0ull, m4 = 0ull;
        if (MODE == 1) {
            m = masks[t * L + g];
            m4 = m14s[t * L + g];
        } else if (MODE == 2) {
            const bool last = g == L - 1;
            m = last ? 0ull : std_t1_mask<B>(false);
            m4 = last ? 0ull : std_t1_mask<B>(true);
        }
        float gx[B], gy[B], gz[B];
#pragma unroll
        for (int b = 0; b < B; ++b)
            partner_x2<B, MASKED>(r, hs, nse, qq, f, posA[sJ + b], posB[sJ + b], dprm[sJ + b], b, m, m4,
                                  s_lj, s_c, gx[b], gy[b], gz[b]);
#pragma unroll
        for (int b = 0; b < B; ++b) hand_over<B>(f, b, gx[b], gy[b], gz[b], gmask, base + src);
    };
    const int TF = (L - 1) / 2;
    // The excluded and scaled 1-4 pairs of a chain lie in the own block and
    // the t = 1 tile: that tile runs the masked code, the others the plain
    // code.  A topology with masked pairs further out (lay.far_masks) runs
    // the masked code on every tile.
    if (TF >= 1) {
        if (lay.std_chain && L >= 3)
            tile(1, std::integral_constant<int, 2>{});
        else
            tile(1, std::integral_constant<int, 1>{});
    }
    if (!lay.far_masks) {
#pragma unroll 1
        for (int t = 2; t <= TF; ++t) tile(t, std::integral_constant<int, 0>{});
    } else {
#pragma unroll 1
        for (int t = 2; t <= TF; ++t) tile(t, std::integral_constant<int, 1>{});
    }
    if ((L & 1) == 0) {
        const int t = L / 2;
        const int J = (g + t) % L;
        const int sJ = J * C::BS;
        float gx[B], gy[B], gz[B];
#pragma unroll
        for (int b = 0; b < B; ++b) gx[b] = gy[b] = gz[b] = 0.f;
        if (g < t) {
            const unsigned long long m = masks[t * L + g], m4 = m14s[t * L + g];
#pragma unroll
            for (int b = 0; b < B; ++b)
                partner_x2<B, true>(r, hs, nse, qq, f, posA[sJ + b], posB[sJ + b], dprm[sJ + b], b,
                                    m, m4, s_lj, s_c, gx[b], gy[b], gz[b]);
        }
        const int src = (g - t + L) % L;
#pragma unroll
        for (int b = 0; b < B; ++b) hand_over<B>(f, b, gx[b], gy[b], gz[b], gmask, base + src);
    }
    // bonded terms; forces on the next block's first atoms go to lane g + 1
    float3 sf[3];
    bonded_chain_x2<B>(sm, lay, prm, posA, posB, L, g, r, f, sf);
    {
        int src = g - 1;
        src = (src < 0) ? src + L : src;  // lane L-1 has no next block and sends zeros
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const float rx = __shfl_sync(gmask, sf[m].x, base + src);
            const float ry = __shfl_sync(gmask, sf[m].y, base + src);
            const float rz = __shfl_sync(gmask, sf[m].z, base + src);
            if (g > 0) f.add(m, rx, ry, rz);
        }
    }
}

// Positions of one atom as partners read them: duplicated and negated.
template <int B>
__device__ __forceinline__ void store_pos_x2(float4* posA, float4* posB, int s, float x, float y,
                                             float z) {
    posA[s] = make_float4(-x, -x, -y, -y);
    *reinterpret_cast<float2*>(&posB[s]) = make_float2(-z, -z);
}

// theta BAOAB steps of replica k by the L lanes of one group.  Velocities
// live in shared memory (vel, {vx, vy, vz, 0} per atom slot) and are touched
// only by the integrator; aux holds {dt/(2m), sqrt((1 - c1^2) k_B T / m)}.
template <int B>
__device__ __forceinline__ void advance_replica_x2(const PropParams& p, const unsigned char* sm,
                                                   const float4* prm, const float4* dprm,
                                                   const float2* aux,
                                                   const unsigned long long* masks, float4* posA,
                                                   float4* posB, float4* vel, long long k, int L,
                                                   int g, int base, unsigned gmask) {
    using C = X2Cfg<B>;
    const TopoLayout& lay = p.lay;
    const int N = lay.n_atoms, Np = lay.n_pad;
    const int s0 = g * C::BS;  // the lane's first atom slot
    const uint32_t step_base = (p.dev_counters ? p.dev_counters[0] : 0u) + p.step0;
    const float* st = p.state_in + (size_t)k * 6 * Np;
    Own<B> r, f, hs, nse, qq;
#pragma unroll
    for (int a = 0; a < B; ++a) {
        const int i = g * B + a;
        const int sl = s0 + a;
        float4 vv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < N) {
            r.set(a, st[i], st[Np + i], st[2 * Np + i]);
            vv = make_float4(st[3 * Np + i], st[4 * Np + i], st[5 * Np + i], 0.f);
        } else {
            const float3 q = far_point(i);
            r.set(a, q.x, q.y, q.z);
        }
        vel[sl] = vv;
        const float4 c = prm[sl];
        hs.set(a, c.x, 0.f, 0.f);
        nse.set(a, -c.y, 0.f, 0.f);
        qq.set(a, c.z, 0.f, 0.f);
        posA[sl] = make_float4(-r.gx(a), -r.gx(a), -r.gy(a), -r.gy(a));
        posB[sl] = make_float4(-r.gz(a), -r.gz(a), c.z, c.z);
    }
    __syncwarp(gmask);
    const float hdt = p.hdt, c1 = p.c1;
    // s = -1 evaluates the forces of the incoming state; s >= 0 are BAOAB
    // steps.  The closing kick of step s - 1 is applied at the start of step
    // s (same operations in the same order as kicking at the end of s - 1).
    for (int s = -1; s < p.theta; ++s) {
        if (s >= 0) {
            const uint32_t step = step_base + (uint32_t)s;
#pragma unroll
            for (int a = 0; a < B; ++a) {
                const int i = g * B + a;
                const int sl = s0 + a;
                const float2 cf = aux[sl];
                float4 vv = vel[sl];
                float x = r.gx(a), y = r.gy(a), z = r.gz(a);
                const float fx = f.gx(a), fy = f.gy(a), fz = f.gz(a);
                if (s > 0) {  // closing B of the previous step
                    vv.x = fmaf(cf.x, fx, vv.x);
                    vv.y = fmaf(cf.x, fy, vv.y);
                    vv.z = fmaf(cf.x, fz, vv.z);
                }
                vv.x = fmaf(cf.x, fx, vv.x);  // B
                vv.y = fmaf(cf.x, fy, vv.y);
                vv.z = fmaf(cf.x, fz, vv.z);
                x = fmaf(hdt, vv.x, x);  // A
                y = fmaf(hdt, vv.y, y);
                z = fmaf(hdt, vv.z, z);
                {  // O (padding atoms: zero noise scale, velocity stays 0)
                    const float3 w = normal3_fast(p.seed, (uint32_t)i, (uint32_t)k, step, p.purpose_mol);
                    vv.x = fmaf(c1, vv.x, cf.y * w.x);
                    vv.y = fmaf(c1, vv.y, cf.y * w.y);
                    vv.z = fmaf(c1, vv.z, cf.y * w.z);
                }
                x = fmaf(hdt, vv.x, x);  // A
                y = fmaf(hdt, vv.y, y);
                z = fmaf(hdt, vv.z, z);
                r.set(a, x, y, z);
                vel[sl] = vv;
            }
            __syncwarp(gmask);  // every lane has finished reading the previous positions
#pragma unroll
            for (int a = 0; a < B; ++a) store_pos_x2<B>(posA, posB, s0 + a, r.gx(a), r.gy(a), r.gz(a));
            __syncwarp(gmask);
        }
        forces_x2<B>(sm, lay, prm, dprm, masks, posA, posB, L, g, base, gmask, r, hs, nse, qq, f);
    }
    // closing B of the last step
    Own<B> v;
#pragma unroll
    for (int a = 0; a < B; ++a) {
        const int sl = s0 + a;
        float4 vv = vel[sl];
        if (p.theta > 0) {
            const float h = aux[sl].x;
            vv.x = fmaf(h, f.gx(a), vv.x);
            vv.y = fmaf(h, f.gy(a), vv.y);
            vv.z = fmaf(h, f.gz(a), vv.z);
        }
        v.set(a, vv.x, vv.y, vv.z);
    }
    // potential energy of the final positions: the scalar energy pass of
    // propagate_impl.cuh on {x, y, z, 0} records in posA
    __syncwarp(gmask);
#pragma unroll
    for (int a = 0; a < B; ++a) posA[g * C::BS + a] = make_float4(r.gx(a), r.gy(a), r.gz(a), 0.f);
    __syncwarp(gmask);
    const double e_acc = energy_pass<B, true>(sm, lay, prm, posA, masks, L, g);

    // write back and per-replica observables
    float* so = p.state_out + (size_t)k * 6 * Np;
    double ek = 0.0, cx = 0.0, cy = 0.0, cz = 0.0;
#pragma unroll
    for (int a = 0; a < B; ++a) {
        const int i = g * B + a;
        if (i < N) {
            const float xa = r.gx(a), ya = r.gy(a), za = r.gz(a);
            const float vxa = v.gx(a), vya = v.gy(a), vza = v.gz(a);
            if (p.theta > 0) {
                so[i] = xa;
                so[Np + i] = ya;
                so[2 * Np + i] = za;
                so[3 * Np + i] = vxa;
                so[4 * Np + i] = vya;
                so[5 * Np + i] = vza;
            }
            if (p.fout) {
                float* fo = p.fout + (size_t)k * 3 * Np;
                fo[i] = f.gx(a);
                fo[Np + i] = f.gy(a);
                fo[2 * Np + i] = f.gz(a);
            }
            const double m = (double)p.masses[i];
            ek += 0.5 * m * ((double)vxa * vxa + (double)vya * vya + (double)vza * vza);
            cx += xa;
            cy += ya;
            cz += za;
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
            const double dx = r.gx(a) - cx, dy = r.gy(a) - cy, dz = r.gz(a) - cz;
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

template <int B>
__global__ void __launch_bounds__(X2Cfg<B>::MAX_THREADS, X2Cfg<B>::MIN_BLOCKS)
    propagate_x2_kernel(const PropParams p) {
    using C = X2Cfg<B>;
    extern __shared__ float4 smem4[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(smem4);
    const TopoLayout& lay = p.lay;
    const int tb = x2_topo_bytes(lay);
    {
        const float4* src = reinterpret_cast<const float4*>(p.topo);
        for (int i = threadIdx.x; i < tb / 16; i += blockDim.x) smem4[i] = src[i];
    }
    __syncthreads();
    const float4* prm = reinterpret_cast<const float4*>(sm + lay.off_params);
    float4* dprm = smem4 + tb / 16;
    float2* aux = reinterpret_cast<float2*>(dprm + lay.nk);
    for (int i = threadIdx.x; i < lay.nk; i += blockDim.x) {
        const float4 c = prm[i];
        dprm[i] = make_float4(c.x, c.x, c.y, c.y);
        aux[i] = make_float2(p.hdt * c.w, p.c2kT * sqrtf(c.w));
    }
    __syncthreads();
    const unsigned long long* masks = reinterpret_cast<const unsigned long long*>(sm + lay.off_masks);
    float4* slots = dprm + lay.nk + (lay.nk + 1) / 2;

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
    float4* posA = slots + slot_local * x2_slot_f4(lay);
    float4* posB = posA + lay.nk;
    float4* vel = posB + lay.nk;

    const long long R = p.live ? (long long)*p.live : p.R;
    for (long long k = (long long)blockIdx.x * rpb + slot_local; k < R;
         k += (long long)gridDim.x * rpb)
        advance_replica_x2<B>(p, sm, prm, dprm, aux, masks, posA, posB, vel, k, L, g, base, gmask);
}

template <int B>
cudaError_t propagate_x2_launch(const PropParams* p, int warps, int grid, size_t smem,
                                cudaStream_t s, int* blocks_per_sm) {
    auto kern = propagate_x2_kernel<B>;
    const cudaError_t e = ensure_dyn_smem((const void*)kern, smem);
    if (e != cudaSuccess) return e;
    if (!p) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, warps * 32, smem);
    kern<<<grid, warps * 32, smem, s>>>(*p);
    return cudaGetLastError();
}

}  // namespace pamd
