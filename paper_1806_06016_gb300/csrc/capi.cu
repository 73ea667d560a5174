// capi.cu -- the extern "C" entry points declared in include/pamd.h.
//
// Host-side runtime: validates the topology, packs it into the table the
// propagate kernel keeps in shared memory (per-atom parameters, 64-bit
// exclusion masks per pair tile, bonded terms split into atom-disjoint colour
// classes), owns the device buffers, chooses the launch shape, and captures a
// whole anneal into one CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pamd_adaptive.h"
#include "../../include/pamd_wham.h"
#include "mlp_internal.h"
#include "pamd_internal.h"

using namespace pamd;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

int cuda_fail(pamd_ctx* c, cudaError_t e, const char* what) {
    if (c) c->broken = true;
    return fail(PAMD_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define PAMD_CU(ctx, call)                                      \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call); \
    } while (0)

void* dalloc(pamd_ctx* c, size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    if (bytes == 0) bytes = 256;
    void* p = nullptr;
    if (c->dev_alloc) {
        p = c->dev_alloc(bytes, c->alloc_user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) c->allocations.push_back(p);
    return p;
}

void free_all(pamd_ctx* c) {
    for (void* p : c->allocations) {
        if (c->dev_free) c->dev_free(p, c->alloc_user);
        else cudaFree(p);
    }
    c->allocations.clear();
}

int round_up(int v, int m) { return (v + m - 1) / m * m; }

bool finite_all(const double* a, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

int check_indices(const int32_t* idx, int n_terms, int arity, int N, const char* what) {
    if (n_terms < 0) return fail(PAMD_EINVAL, std::string(what) + ": negative count");
    if (n_terms > 0 && !idx) return fail(PAMD_EINVAL, std::string(what) + ": null index array");
    for (int t = 0; t < n_terms; ++t) {
        for (int a = 0; a < arity; ++a) {
            const int i = idx[t * arity + a];
            if (i < 0 || i >= N) return fail(PAMD_EINVAL, std::string(what) + ": atom index out of range");
            for (int b = 0; b < a; ++b)
                if (idx[t * arity + b] == i)
                    return fail(PAMD_EINVAL, std::string(what) + ": repeated atom in one term");
        }
    }
    return PAMD_OK;
}

// Greedy colouring: term t gets the smallest colour whose atoms it does not
// touch.  Returns the permutation that sorts terms by colour and the colour
// start offsets.
int colour_terms(const std::vector<std::vector<int>>& atoms, int N, std::vector<int>& order,
                 std::vector<int>& starts, int* n_colors) {
    const int n = (int)atoms.size();
    std::vector<int> col(n, -1);
    std::vector<std::vector<char>> used;
    int nc = 0;
    for (int t = 0; t < n; ++t) {
        int c = 0;
        for (;; ++c) {
            if (c == nc) {
                used.emplace_back(N, 0);
                ++nc;
            }
            bool ok = true;
            for (int i : atoms[t])
                if (used[c][i]) ok = false;
            if (ok) break;
        }
        if (c >= kMaxColors) return fail(PAMD_EUNSUPPORTED, "bonded terms need more than 64 colour classes");
        col[t] = c;
        for (int i : atoms[t]) used[c][i] = 1;
    }
    order.resize(n);
    for (int t = 0; t < n; ++t) order[t] = t;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return col[a] < col[b]; });
    starts.assign(kMaxColors + 1, n);
    for (int c = 0; c <= nc; ++c) {
        int s = 0;
        while (s < n && col[order[s]] < c) ++s;
        starts[c] = s;
    }
    *n_colors = nc;
    return PAMD_OK;
}

// Launch shape: B atoms per lane (1..8), L = ceil(N/B) lanes per replica
// (<= 32), G = floor(32/L) replicas per warp.  The cost of one replica-step per
// warp slot is modelled as (pair evaluations per lane + per-atom work) / G,
// with the per-atom work (bonded terms, noise, integration) taken as 16 pair
// evaluations; the cheapest shape is chosen.
int choose_lanes(int N, int requested, int* L, int* B) {
    if (requested) {
        if (requested < 1 || requested > 32) return fail(PAMD_EINVAL, "lanes_per_replica must be 0..32");
        *L = requested;
        *B = (N + requested - 1) / requested;
        if (*B > 8) return fail(PAMD_EINVAL, "lanes_per_replica too small for this molecule (8 atoms per lane at most)");
        *L = (N + *B - 1) / *B;  // no lane without atoms
        return PAMD_OK;
    }
    double best = 1e300;
    for (int b = 1; b <= 8; ++b) {
        const int l = (N + b - 1) / b;
        if (l > 32) continue;
        const int G = 32 / l;
        const double cost = (0.5 * b * (double)(l * b) + 16.0 * b) / G;
        if (cost < best) {
            best = cost;
            *L = l;
            *B = b;
        }
    }
    if (best == 1e300) return fail(PAMD_EUNSUPPORTED, "molecule too large");
    return PAMD_OK;
}

// True when the bonded lists are those of a linear chain: bond k = (k, k+1),
// angle k = (k, k+1, k+2), dihedral k = (k..k+3) (either direction), one
// entry per k, and the 1-4 pairs are exactly {(k, k+3)}.
bool is_linear_chain(const pamd_topology* t) {
    const int N = t->n_atoms;
    auto run = [](const int32_t* idx, int n, int arity, int k) {
        bool fwd = true, bwd = true;
        for (int a = 0; a < arity; ++a) {
            fwd = fwd && idx[k * arity + a] == k + a;
            bwd = bwd && idx[k * arity + a] == k + arity - 1 - a;
        }
        return fwd || bwd;
    };
    if (t->n_bonds != std::max(N - 1, 0) || t->n_angles != std::max(N - 2, 0) ||
        t->n_dihedrals != std::max(N - 3, 0) || t->n_pair14 != std::max(N - 3, 0))
        return false;
    for (int k = 0; k < t->n_bonds; ++k) if (!run(t->bond, t->n_bonds, 2, k)) return false;
    for (int k = 0; k < t->n_angles; ++k) if (!run(t->angle, t->n_angles, 3, k)) return false;
    for (int k = 0; k < t->n_dihedrals; ++k) if (!run(t->dihedral, t->n_dihedrals, 4, k)) return false;
    std::vector<char> seen(std::max(N - 3, 0), 0);
    for (int p = 0; p < t->n_pair14; ++p) {
        const int i = std::min(t->pair14[2 * p], t->pair14[2 * p + 1]);
        const int j = std::max(t->pair14[2 * p], t->pair14[2 * p + 1]);
        if (j != i + 3 || seen[i]) return false;
        seen[i] = 1;
    }
    // a 1-4 pair that is also excluded would be skipped by the generic path
    for (int p = 0; p < t->n_excl; ++p) {
        const int i = t->excl[2 * p], j = t->excl[2 * p + 1];
        if (std::abs(i - j) == 3) return false;
    }
    return true;
}

// Build the shared-memory table of the propagate kernel.
int build_topology(const pamd_topology* t, int lanes_req, TopoLayout* lay_out,
                   std::vector<unsigned char>& blob) {
    const int N = t->n_atoms;
    if (N < 1) return fail(PAMD_EINVAL, "n_atoms must be >= 1");
    if (N > PAMD_MAX_ATOMS) return fail(PAMD_EUNSUPPORTED, "n_atoms exceeds PAMD_MAX_ATOMS");
    if (!t->mass || !t->charge || !t->sigma || !t->epsilon || !t->x0)
        return fail(PAMD_EINVAL, "null per-atom array");
    if (!finite_all(t->mass, N) || !finite_all(t->charge, N) || !finite_all(t->sigma, N) ||
        !finite_all(t->epsilon, N) || !finite_all(t->x0, 3 * N))
        return fail(PAMD_EINVAL, "non-finite per-atom value");
    for (int i = 0; i < N; ++i) {
        if (!(t->mass[i] > 0)) return fail(PAMD_EINVAL, "masses must be > 0");
        if (t->sigma[i] < 0 || t->epsilon[i] < 0) return fail(PAMD_EINVAL, "sigma and epsilon must be >= 0");
    }
    int rc;
    if ((rc = check_indices(t->bond, t->n_bonds, 2, N, "bonds"))) return rc;
    if ((rc = check_indices(t->angle, t->n_angles, 3, N, "angles"))) return rc;
    if ((rc = check_indices(t->dihedral, t->n_dihedrals, 4, N, "dihedrals"))) return rc;
    if ((rc = check_indices(t->excl, t->n_excl, 2, N, "exclusions"))) return rc;
    if ((rc = check_indices(t->pair14, t->n_pair14, 2, N, "1-4 pairs"))) return rc;
    if (t->n_bonds > 0 && (!t->bond_r0 || !t->bond_k || !finite_all(t->bond_r0, t->n_bonds) ||
                           !finite_all(t->bond_k, t->n_bonds)))
        return fail(PAMD_EINVAL, "bond parameters");
    if (t->n_angles > 0 && (!t->angle_t0 || !t->angle_k || !finite_all(t->angle_t0, t->n_angles) ||
                            !finite_all(t->angle_k, t->n_angles)))
        return fail(PAMD_EINVAL, "angle parameters");
    if (t->n_dihedrals > 0) {
        if (!t->dih_n || !t->dih_k || !t->dih_phase || !finite_all(t->dih_k, t->n_dihedrals) ||
            !finite_all(t->dih_phase, t->n_dihedrals))
            return fail(PAMD_EINVAL, "dihedral parameters");
        for (int d = 0; d < t->n_dihedrals; ++d)
            if (t->dih_n[d] < 1 || t->dih_n[d] > 6) return fail(PAMD_EINVAL, "dihedral multiplicity must be 1..6");
    }
    if (!std::isfinite(t->scale14_lj) || !std::isfinite(t->scale14_coul))
        return fail(PAMD_EINVAL, "1-4 scale factors");

    int L, B;
    if ((rc = choose_lanes(N, lanes_req, &L, &B))) return rc;
    TopoLayout& lay = *lay_out;
    lay = TopoLayout{};
    lay.n_atoms = N;
    lay.n_pad = round_up(N, 4);
    lay.lanes = L;
    lay.per_lane = B;
    lay.block_stride = (B % 2 == 1) ? B : B + 1;
    lay.nk = L * lay.block_stride;
    auto slot = [&](int i) { return (i / B) * lay.block_stride + i % B; };

    // pair kinds: exclusions win over 1-4 entries
    std::vector<char> excl((size_t)N * N, 0);
    for (int p = 0; p < t->n_excl; ++p) {
        const int i = t->excl[2 * p], j = t->excl[2 * p + 1];
        excl[(size_t)i * N + j] = excl[(size_t)j * N + i] = 1;
    }
    std::vector<std::pair<int, int>> p14;
    for (int p = 0; p < t->n_pair14; ++p) {
        const int i = t->pair14[2 * p], j = t->pair14[2 * p + 1];
        if (!excl[(size_t)i * N + j]) p14.emplace_back(i, j);
    }
    // tile masks
    const int TH = L / 2;
    // masks: every pair left out of the plain nonbonded sum (excluded or
    // scaled 1-4); m14: the scaled 1-4 pairs among them
    std::vector<unsigned long long> masks((size_t)(TH + 1) * L, 0ull), m14((size_t)(TH + 1) * L, 0ull);
    auto mask_pair = [&](int i, int j, std::vector<unsigned long long>& mk) {
        const int gi = i / B, gj = j / B, ai = i % B, aj = j % B;
        if (gi == gj) {
            const int a = std::min(ai, aj), b = std::max(ai, aj);
            mk[gi] |= 1ull << (a * B + b);
            return;
        }
        const int tt = ((gj - gi) % L + L) % L;
        if (2 * tt < L || (2 * tt == L && gi < tt)) {
            mk[(size_t)tt * L + gi] |= 1ull << (ai * B + aj);
        } else {
            const int t2 = L - tt;
            mk[(size_t)t2 * L + gj] |= 1ull << (aj * B + ai);
        }
    };
    for (int p = 0; p < t->n_excl; ++p) mask_pair(t->excl[2 * p], t->excl[2 * p + 1], masks);
    for (auto& q : p14) {
        mask_pair(q.first, q.second, masks);
        mask_pair(q.first, q.second, m14);
    }

    // bonded records, coloured
    std::vector<BondRec> bonds;
    std::vector<AngleRec> angles;
    std::vector<DihRec> dihs;
    std::vector<Pair14Rec> prs;
    std::vector<int> starts[4];
    {
        std::vector<std::vector<int>> at;
        for (int b = 0; b < t->n_bonds; ++b) at.push_back({t->bond[2 * b], t->bond[2 * b + 1]});
        std::vector<int> order;
        if ((rc = colour_terms(at, N, order, starts[0], &lay.n_colors[0]))) return rc;
        for (int o : order)
            bonds.push_back({slot(t->bond[2 * o]), slot(t->bond[2 * o + 1]), (float)t->bond_r0[o],
                             (float)t->bond_k[o]});
    }
    {
        std::vector<std::vector<int>> at;
        for (int a = 0; a < t->n_angles; ++a)
            at.push_back({t->angle[3 * a], t->angle[3 * a + 1], t->angle[3 * a + 2]});
        std::vector<int> order;
        if ((rc = colour_terms(at, N, order, starts[1], &lay.n_colors[1]))) return rc;
        for (int o : order)
            angles.push_back({slot(t->angle[3 * o]), slot(t->angle[3 * o + 1]),
                              slot(t->angle[3 * o + 2]), 0, (float)t->angle_t0[o],
                              (float)t->angle_k[o], 0.f, 0.f});
    }
    {
        std::vector<std::vector<int>> at;
        for (int d = 0; d < t->n_dihedrals; ++d)
            at.push_back({t->dihedral[4 * d], t->dihedral[4 * d + 1], t->dihedral[4 * d + 2],
                          t->dihedral[4 * d + 3]});
        std::vector<int> order;
        if ((rc = colour_terms(at, N, order, starts[2], &lay.n_colors[2]))) return rc;
        for (int o : order)
            dihs.push_back({slot(t->dihedral[4 * o]), slot(t->dihedral[4 * o + 1]),
                            slot(t->dihedral[4 * o + 2]), slot(t->dihedral[4 * o + 3]),
                            (float)t->dih_k[o], (float)t->dih_n[o], (float)std::cos(t->dih_phase[o]),
                            (float)std::sin(t->dih_phase[o])});
    }
    {
        std::vector<std::vector<int>> at;
        for (auto& q : p14) at.push_back({q.first, q.second});
        std::vector<int> order;
        if ((rc = colour_terms(at, N, order, starts[3], &lay.n_colors[3]))) return rc;
        for (int o : order)
            prs.push_back({slot(p14[o].first), slot(p14[o].second), (float)t->scale14_lj,
                           (float)t->scale14_coul});
    }
    const bool chain = B >= 3 && is_linear_chain(t);
    lay.chain = chain ? 1 : 0;
    lay.s14_lj = (float)t->scale14_lj;
    lay.s14_c = (float)t->scale14_coul;
    lay.n_bonds = (int)bonds.size();
    lay.n_angles = (int)angles.size();
    lay.n_dihs = (int)dihs.size();
    lay.n_p14 = (int)prs.size();

    int off = 0;
    lay.off_params = off; off += round_up(lay.nk * 16, 16);
    lay.off_masks = off; off += round_up((int)masks.size() * 8, 16);
    lay.off_m14 = off; off += round_up((int)m14.size() * 8, 16);
    lay.far_masks = 0;
    for (size_t q = 2 * (size_t)L; q < masks.size(); ++q)
        if (masks[q]) lay.far_masks = 1;
    // the usual chain exclusions only: the kernels may then leave the own
    // block's 1-2 and 1-3 pairs out by position instead of by mask
    lay.std_chain = 0;
    if (chain) {
        bool std_excl = true;
        for (int i = 0; i < N && std_excl; ++i)
            for (int j = i + 1; j < N; ++j) {
                const bool ex = excl[(size_t)i * N + j] != 0;
                if (ex != (j - i <= 2)) {
                    std_excl = false;
                    break;
                }
            }
        lay.std_chain = std_excl ? 1 : 0;
    }
    lay.off_bonds = off; off += round_up(lay.n_bonds * 16, 16);
    lay.off_angles = off; off += round_up(lay.n_angles * 32, 16);
    lay.off_dihs = off; off += round_up(lay.n_dihs * 32, 16);
    lay.off_p14 = off; off += round_up(lay.n_p14 * 16, 16);
    lay.off_colors = off; off += round_up(4 * (kMaxColors + 1) * 4, 16);
    // chain term parameters, indexed by the term's first atom; one entry per
    // atom slot of the lanes (L B), zero beyond the chain's last term, so that
    // the packed kernel can evaluate every lane's terms without branches
    const int n_slots = std::max(L * B, N);
    lay.off_cbond = off; off += round_up(n_slots * 8, 16);
    lay.off_cangle = off; off += round_up(n_slots * 8, 16);
    lay.off_cdih = off; off += round_up(n_slots * 16, 16);
    // pair-parameter table of the half-ring tiles (chain layouts, when small)
    const size_t tab_bytes = (size_t)TH * B * B * L * 16;
    if (chain && TH > 0 && tab_bytes <= kPairTableMaxBytes) {
        lay.ptab = 1;
        lay.off_ptab = off;
        off += (int)tab_bytes;
    }
    lay.bytes = off;
    blob.assign(off, 0);
    float* prm = reinterpret_cast<float*>(blob.data() + lay.off_params);
    const double sqrt_ke = std::sqrt(kCoulomb);
    for (int i = 0; i < N; ++i) {
        float* q = prm + 4 * slot(i);
        q[0] = (float)(0.5 * t->sigma[i]);
        q[1] = (float)std::sqrt(24.0 * t->epsilon[i]);
        q[2] = (float)(t->charge[i] * sqrt_ke);
        q[3] = (float)(1.0 / t->mass[i]);
    }
    std::memcpy(blob.data() + lay.off_masks, masks.data(), masks.size() * 8);
    std::memcpy(blob.data() + lay.off_m14, m14.data(), m14.size() * 8);
    if (lay.ptab) {
        // the FP32 products the kernel's mixing would form, so both paths agree bitwise
        float* tb = reinterpret_cast<float*>(blob.data() + lay.off_ptab);
        for (int t = 1; t <= TH; ++t)
            for (int g = 0; g < L; ++g) {
                const int J = (g + t) % L;
                for (int b = 0; b < B; ++b)
                    for (int a = 0; a < B; ++a) {
                        const float* pi = prm + 4 * (g * lay.block_stride + a);
                        const float* pj = prm + 4 * (J * lay.block_stride + b);
                        const float sg = pi[0] + pj[0];
                        float* e = tb + 4 * ((((size_t)(t - 1) * B * B + (size_t)b * B + a) * L) + g);
                        e[0] = sg * sg;
                        e[1] = pi[1] * pj[1];
                        e[2] = pi[2] * pj[2];
                        e[3] = e[1] + e[1];  // 2 eps_ij, exact
                    }
            }
    }
    if (!bonds.empty()) std::memcpy(blob.data() + lay.off_bonds, bonds.data(), bonds.size() * 16);
    if (!angles.empty()) std::memcpy(blob.data() + lay.off_angles, angles.data(), angles.size() * 32);
    if (!dihs.empty()) std::memcpy(blob.data() + lay.off_dihs, dihs.data(), dihs.size() * 32);
    if (!prs.empty()) std::memcpy(blob.data() + lay.off_p14, prs.data(), prs.size() * 16);
    if (chain) {
        // per-term parameters indexed by the term's first (lowest) atom
        float* cb = reinterpret_cast<float*>(blob.data() + lay.off_cbond);
        for (int b = 0; b < t->n_bonds; ++b) {
            const int d = std::min(t->bond[2 * b], t->bond[2 * b + 1]);
            cb[2 * d] = (float)t->bond_r0[b];
            cb[2 * d + 1] = (float)t->bond_k[b];
        }
        float* ca = reinterpret_cast<float*>(blob.data() + lay.off_cangle);
        for (int a = 0; a < t->n_angles; ++a) {
            const int d = std::min(t->angle[3 * a], t->angle[3 * a + 2]);
            ca[2 * d] = (float)t->angle_t0[a];
            ca[2 * d + 1] = (float)t->angle_k[a];
        }
        float* cd = reinterpret_cast<float*>(blob.data() + lay.off_cdih);
        for (int h = 0; h < t->n_dihedrals; ++h) {
            const int d = std::min(t->dihedral[4 * h], t->dihedral[4 * h + 3]);
            cd[4 * d] = (float)t->dih_k[h];
            cd[4 * d + 1] = (float)t->dih_n[h];
            cd[4 * d + 2] = (float)std::cos(t->dih_phase[h]);
            cd[4 * d + 3] = (float)std::sin(t->dih_phase[h]);
        }
    }
    int* cols = reinterpret_cast<int*>(blob.data() + lay.off_colors);
    for (int ty = 0; ty < 4; ++ty)
        for (int q = 0; q <= kMaxColors; ++q) cols[ty * (kMaxColors + 1) + q] = starts[ty][q];
    return PAMD_OK;
}

cudaError_t propagate_dispatch_any(const TopoLayout& lay, const PropParams* p, int warps, int grid,
                                   size_t smem, cudaStream_t s, int* occ) {
    const bool chain = lay.chain != 0;
    const bool table = lay.ptab != 0;
    if (lay.packed) return propagate_x2_dispatch(lay.per_lane, p, warps, grid, smem, s, occ);
    if (lay.paired) {
        switch (lay.per_lane) {
            case 2: return propagate2_b2(p, chain, warps, grid, smem, s, occ);
            case 3: return propagate2_b3(p, chain, warps, grid, smem, s, occ);
            case 4: return propagate2_b4(p, chain, warps, grid, smem, s, occ);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (lay.per_lane) {
        case 1: return propagate_b1(p, chain, table, warps, grid, smem, s, occ);
        case 2: return propagate_b2(p, chain, table, warps, grid, smem, s, occ);
        case 3: return propagate_b3(p, chain, table, warps, grid, smem, s, occ);
        case 4: return propagate_b4(p, chain, table, warps, grid, smem, s, occ);
        case 5: return propagate_b5(p, chain, table, warps, grid, smem, s, occ);
        case 6: return propagate_b6(p, chain, table, warps, grid, smem, s, occ);
        case 7: return propagate_b7(p, chain, table, warps, grid, smem, s, occ);
        case 8: return propagate_b8(p, chain, table, warps, grid, smem, s, occ);
        default: return cudaErrorInvalidValue;
    }
}

// float4s of shared memory per replica slot (single, packed) or replica-pair
// slot (paired)
int slot_f4(const TopoLayout& lay) {
    if (lay.packed) return x2_slot_f4(lay);
    return lay.paired ? 3 * lay.nk + 1 : 2 * lay.nk + 1;
}

// Shared memory of one propagate block with `units` replica (or replica-pair)
// slots: the topology table (for the packed kernel without the pair table,
// with its per-atom tables), then the slots.
size_t prop_smem_units(const TopoLayout& lay, int units) {
    const size_t table = lay.packed ? (size_t)x2_topo_bytes(lay) + (size_t)x2_table_f4(lay) * 16
                                    : (size_t)lay.bytes;
    return table + (size_t)units * slot_f4(lay) * 16;
}

size_t prop_smem(const pamd_ctx* c) {
    return prop_smem_units(c->lay, c->lay.paired ? c->rpb / 2 : c->rpb);
}

float* cur_state(pamd_ctx* c) { return c->cur_is_alt ? c->b.state_alt : c->b.state; }
bool is_f64(const pamd_ctx* c) { return c->precision == PAMD_PREC_FP64; }
// bytes of one population buffer: 6 Np values per replica, FP32 or FP64
size_t state_bytes(const pamd_ctx* c) {
    return (is_f64(c) ? sizeof(double) : sizeof(float)) * 6 * (size_t)c->Np * (size_t)c->R;
}
double* cur_E(pamd_ctx* c) { return c->cur_is_alt ? c->b.E_alt : c->b.E; }
int32_t* cur_fam(pamd_ctx* c) { return c->cur_is_alt ? c->b.fam_alt : c->b.fam; }

void fill_prop_params(pamd_ctx* c, PropParams& p, float* state, double* E, double* ke, double* rg,
                      int theta, double dt, double T, const uint32_t* dev_ctr, uint32_t step0,
                      float* fout);

int launch_prop_on(pamd_ctx* c, float* state, double* E, double* ke, double* rg, int theta,
                   double dt, double T, const uint32_t* dev_ctr, uint32_t step0, float* fout) {
    if (is_f64(c)) {
        cudaError_t e = launch_propagate_f64(c, reinterpret_cast<double*>(state), E, ke, rg, theta,
                                             dt, T, dev_ctr, step0, reinterpret_cast<double*>(fout));
        if (e != cudaSuccess) return cuda_fail(c, e, "propagate launch (FP64)");
        return PAMD_OK;
    }
    if (c->mlp) {
        const int rc = mlp_propagate(c->mlp, state, E, ke, rg, fout, c->b.masses, &c->b.scal->status,
                                     dev_ctr, c->R, c->Np, theta, dt, T, c->gamma, c->seed, step0,
                                     kPurposeNoise | ((uint32_t)c->mol << 8), c->stream, &c->launches);
        if (rc == PAMD_ECUDA) c->broken = true;
        return rc;
    }
    PropParams p{};
    fill_prop_params(c, p, state, E, ke, rg, theta, dt, T, dev_ctr, step0, fout);
    cudaError_t e = propagate_dispatch_any(c->lay, &p, c->warps_per_block, c->grid_prop,
                                           prop_smem(c), c->stream, nullptr);
    c->launches += 1;
    if (e != cudaSuccess) return cuda_fail(c, e, "propagate launch");
    return PAMD_OK;
}

void fill_prop_params(pamd_ctx* c, PropParams& p, float* state, double* E, double* ke, double* rg,
                      int theta, double dt, double T, const uint32_t* dev_ctr, uint32_t step0,
                      float* fout) {
    p.state_in = state;
    p.state_out = state;
    p.E = E;
    p.ke = ke;
    p.rg = rg;
    p.fout = fout;
    p.masses = c->b.masses;
    p.topo = c->b.topo;
    p.status = &c->b.scal->status;
    p.dev_counters = dev_ctr;
    p.live = c->variable ? c->b.counters + 2 : nullptr;
    p.lay = c->lay;
    p.R = c->R;
    p.theta = theta;
    p.hdt = (float)(0.5 * dt);
    const double c1 = std::exp(-c->gamma * dt);
    p.c1 = (float)c1;
    p.c2kT = (float)std::sqrt((1.0 - c1 * c1) * kBoltzmann * T);
    p.seed = c->seed;
    p.step0 = step0;
    p.purpose_mol = kPurposeNoise | ((uint32_t)c->mol << 8);
}

int launch_prop(pamd_ctx* c, int theta, double dt, double T, const uint32_t* dev_ctr,
                uint32_t step0, float* fout) {
    return launch_prop_on(c, cur_state(c), cur_E(c), c->b.ke, c->b.rg, theta, dt, T, dev_ctr,
                          step0, fout);
}

// Device tables of the all-FP64 mode: one allocation, laid out on the host.
int build_topo_f64(pamd_ctx* c, const pamd_topology* t, std::vector<unsigned char>& blob) {
    const int N = t->n_atoms, Np = c->Np;
    std::vector<double> sh(N), ep(N), q(N), im(N), x0(3 * (size_t)Np, 0.0);
    double com[3] = {0, 0, 0}, mt = 0;
    for (int i = 0; i < N; ++i) {
        sh[i] = 0.5 * t->sigma[i];
        ep[i] = t->epsilon[i];
        q[i] = t->charge[i];
        im[i] = 1.0 / t->mass[i];
        for (int k = 0; k < 3; ++k) com[k] += t->mass[i] * t->x0[3 * i + k];
        mt += t->mass[i];
    }
    for (int i = 0; i < N; ++i)
        for (int k = 0; k < 3; ++k) x0[(size_t)k * Np + i] = t->x0[3 * i + k] - com[k] / mt;
    std::vector<unsigned char> kind((size_t)N * N, 0);
    for (int p = 0; p < t->n_pair14; ++p) {
        const int i = t->pair14[2 * p], j = t->pair14[2 * p + 1];
        kind[(size_t)i * N + j] = kind[(size_t)j * N + i] = 2;
    }
    for (int p = 0; p < t->n_excl; ++p) {
        const int i = t->excl[2 * p], j = t->excl[2 * p + 1];
        kind[(size_t)i * N + j] = kind[(size_t)j * N + i] = 1;
    }
    std::vector<double> bp(2 * (size_t)t->n_bonds), ap(2 * (size_t)t->n_angles), dp(4 * (size_t)t->n_dihedrals);
    for (int b = 0; b < t->n_bonds; ++b) { bp[2 * b] = t->bond_r0[b]; bp[2 * b + 1] = t->bond_k[b]; }
    for (int a = 0; a < t->n_angles; ++a) { ap[2 * a] = t->angle_t0[a]; ap[2 * a + 1] = t->angle_k[a]; }
    for (int d = 0; d < t->n_dihedrals; ++d) {
        dp[4 * d] = t->dih_k[d];
        dp[4 * d + 1] = (double)t->dih_n[d];
        dp[4 * d + 2] = std::cos(t->dih_phase[d]);
        dp[4 * d + 3] = std::sin(t->dih_phase[d]);
    }
    // append each array 16-byte aligned and remember its offset
    std::vector<size_t> off;
    auto put = [&](const void* src, size_t bytes) {
        const size_t o = (blob.size() + 15) & ~size_t(15);
        blob.resize(o + bytes);
        if (bytes) std::memcpy(blob.data() + o, src, bytes);
        off.push_back(o);
    };
    put(sh.data(), 8 * sh.size()); put(ep.data(), 8 * ep.size()); put(q.data(), 8 * q.size());
    put(im.data(), 8 * im.size()); put(x0.data(), 8 * x0.size()); put(kind.data(), kind.size());
    put(t->bond, 8 * (size_t)t->n_bonds); put(bp.data(), 8 * bp.size());
    put(t->angle, 12 * (size_t)t->n_angles); put(ap.data(), 8 * ap.size());
    put(t->dihedral, 16 * (size_t)t->n_dihedrals); put(dp.data(), 8 * dp.size());
    unsigned char* d = (unsigned char*)dalloc(c, blob.size() + 16);
    if (!d) return fail(PAMD_ENOMEM, "FP64 tables");
    c->top64_blob = d;
    TopoF64& T = c->top64;
    T.n_atoms = N;
    T.sigma_half = (const double*)(d + off[0]);
    T.epsilon = (const double*)(d + off[1]);
    T.charge = (const double*)(d + off[2]);
    T.inv_mass = (const double*)(d + off[3]);
    T.x0 = (const double*)(d + off[4]);
    T.kind = d + off[5];
    T.s14_lj = t->scale14_lj;
    T.s14_c = t->scale14_coul;
    T.n_bonds = t->n_bonds;
    T.n_angles = t->n_angles;
    T.n_dihs = t->n_dihedrals;
    T.bond = (const int*)(d + off[6]);
    T.bond_p = (const double*)(d + off[7]);
    T.angle = (const int*)(d + off[8]);
    T.angle_p = (const double*)(d + off[9]);
    T.dih = (const int*)(d + off[10]);
    T.dih_p = (const double*)(d + off[11]);
    return PAMD_OK;
}

// In-process cache of tuned shapes, mirrored to the file named by
// PAMD_TUNE_CACHE ("N R chain lanes_req -> L warps" per line).
struct TuneKey {
    int N;
    long long R;
    int chain;
    int lanes_req;
    int pair_arith;
};
struct TuneShape {
    int L, W, variant;  // variant: kVarScalar, kVarPaired or kVarPacked
};
// Shapes a tuning run may choose: atoms per lane bmin..bmax, the given warp
// counts, two-replica kernels or not, packed-pair kernels or not.  The batched
// kernel needs B = 3..7, kBatchThreads / 32 warps, single replicas and
// scalar pair arithmetic.
struct TuneLimits {
    int bmin, bmax;
    bool paired_ok;
    bool packed_ok;
    std::vector<int> warps;
    int key_tag;  // separates the cache entries of restricted searches
};
int autotune_with(pamd_ctx* c, int32_t theta_probe, const TuneLimits& lim, pamd_tune* out);
std::mutex g_tune_mu;
std::vector<std::pair<TuneKey, TuneShape>> g_tune;

bool tune_cache_lookup(const TuneKey& k, TuneShape* out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto match = [&](const TuneKey& q) {
        return q.N == k.N && q.R == k.R && q.chain == k.chain && q.lanes_req == k.lanes_req &&
               q.pair_arith == k.pair_arith;
    };
    for (auto& e : g_tune)
        if (match(e.first)) {
            *out = e.second;
            return true;
        }
    const char* path = std::getenv("PAMD_TUNE_CACHE");
    if (!path || !*path) return false;
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    TuneKey q;
    TuneShape t;
    bool found = false;
    while (std::fscanf(f, "%d %lld %d %d %d %d %d %d", &q.N, &q.R, &q.chain, &q.lanes_req,
                       &q.pair_arith, &t.L, &t.W, &t.variant) == 8) {
        if (match(q) && t.L >= 1 && t.L <= 32 && (t.W == 2 || t.W == 4 || t.W == 8) &&
            (t.variant == kVarScalar || t.variant == kVarPaired || t.variant == kVarPacked)) {
            *out = t;
            found = true;
        }
    }
    std::fclose(f);
    if (found) g_tune.push_back({k, *out});
    return found;
}

void tune_cache_store(const TuneKey& k, const TuneShape& t) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.push_back({k, t});
    const char* path = std::getenv("PAMD_TUNE_CACHE");
    if (!path || !*path) return;
    if (FILE* f = std::fopen(path, "a")) {
        std::fprintf(f, "%d %lld %d %d %d %d %d %d\n", k.N, k.R, k.chain, k.lanes_req, k.pair_arith,
                     t.L, t.W, t.variant);
        std::fclose(f);
    }
}

// Warps per block (<= requested, shared memory permitting), replicas per
// block and the persistent grid for layout `lay`.
// True when the packed-pair kernel can run layout `lay`.
bool packed_ok(const TopoLayout& lay) { return lay.chain && lay.per_lane >= 3 && lay.per_lane <= 8; }

int set_launch_shape(pamd_ctx* c, const TopoLayout& lay_in, int warps_req, int variant) {
    TopoLayout lay = lay_in;
    lay.paired = variant == kVarPaired ? 1 : 0;
    lay.packed = variant == kVarPacked ? 1 : 0;
    if (lay.paired && (lay.per_lane < 2 || lay.per_lane > 4))
        return fail(PAMD_EUNSUPPORTED, "two replicas per lane need 2..4 atoms per lane");
    if (lay.packed && !packed_ok(lay))
        return fail(PAMD_EUNSUPPORTED, "packed pair arithmetic needs a linear chain with 3..8 atoms per lane");
    int dev = 0, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int groups_per_warp = 32 / lay.lanes;  // idle lanes when L does not divide 32
    int warps = warps_req ? warps_req : 4;
    // the single-replica kernel of some atoms-per-lane counts takes smaller blocks
    if (lay.packed)
        warps = std::min(warps, kPackedMaxThreads / 32);
    else if (!lay.paired && lay.per_lane >= 1 && lay.per_lane <= 8)
        warps = std::min(warps, prop_max_threads(lay.per_lane) / 32);
    auto smem = [&](int w) { return (long long)prop_smem_units(lay, w * groups_per_warp); };
    while (smem(warps) > max_smem && warps > 1) --warps;
    if (smem(warps) > max_smem) return fail(PAMD_EUNSUPPORTED, "molecule tables exceed shared memory");
    int occ = 0;
    cudaError_t e = propagate_dispatch_any(lay, nullptr, warps, 0, (size_t)smem(warps), nullptr, &occ);
    if (e != cudaSuccess || occ < 1)
        return fail(PAMD_ECUDA, std::string("propagate occupancy: ") + cudaGetErrorString(e));
    c->lay = lay;
    c->warps_per_block = warps;
    c->rpb = warps * groups_per_warp * (lay.paired ? 2 : 1);
    const long long batches = (c->R + c->rpb - 1) / c->rpb;
    c->grid_prop = (int)std::min<long long>(batches, (long long)c->num_sms * occ);
    return PAMD_OK;
}

bool is_batch(const pamd_ctx* c) { return !c->subs.empty(); }

// One launch of the batched kernel per group (atoms per lane, pair
// arithmetic), the groups on streams of their own forked from and joined back
// to the context's stream (parallel branches when the anneal is captured as
// a graph), so that one group's last work items overlap the next group's
// instead of idling SMs.
// graph: counters come from each molecule's device counters plus step_off.
int launch_prop_batch(pamd_ctx* c, int theta, double dt, double T, bool graph, uint32_t step_off) {
    BatchParams bp{};
    for (size_t m = 0; m < c->subs.size(); ++m) {
        pamd_ctx* s = c->subs[m];
        fill_prop_params(s, bp.mol[m], cur_state(s), cur_E(s), s->b.ke, s->b.rg, theta, dt, T,
                         graph ? s->b.counters : nullptr, graph ? step_off : s->step, nullptr);
    }
    PAMD_CU(c, cudaMemsetAsync(c->queue, 0, sizeof(int) * c->groups.size(), c->stream));
    const bool fork = c->groups.size() > 1 && c->group_streams.size() == c->groups.size();
    if (fork) PAMD_CU(c, cudaEventRecord(c->fork_event, c->stream));
    for (size_t q = 0; q < c->groups.size(); ++q) {
        const pamd_ctx::BatchGroup& gr = c->groups[q];
        bp.n_items = gr.n_items;
        bp.items = c->items + gr.first_item;
        bp.queue = c->queue + q;
        cudaStream_t s = fork ? c->group_streams[q] : c->stream;
        if (fork) PAMD_CU(c, cudaStreamWaitEvent(s, c->fork_event, 0));
        const cudaError_t e = gr.packed ? launch_propagate_batch_x2(bp, gr.B, gr.grid, gr.smem, s)
                                        : launch_propagate_batch(bp, gr.B, gr.grid, gr.smem, s);
        c->launches += 1;
        if (e != cudaSuccess) return cuda_fail(c, e, "batched propagate launch");
        if (fork) {
            PAMD_CU(c, cudaEventRecord(c->group_events[q], s));
            PAMD_CU(c, cudaStreamWaitEvent(c->stream, c->group_events[q], 0));
        }
    }
    return PAMD_OK;
}

// Atoms per lane of a molecule in a batch: the cost-model choice kept in the
// batched kernel's range 3..7.
int batch_lanes(int N) {
    int L = 0, B = 0;
    if (choose_lanes(N, 0, &L, &B)) return 0;
    B = std::min(7, std::max(3, B));
    return (N + B - 1) / B;
}

int check_ctx(pamd_ctx* c) {
    if (!c) return fail(PAMD_EINVAL, "null context");
    if (c->broken) return fail(PAMD_ESTATE, "context broken by an earlier CUDA failure");
    return PAMD_OK;
}

int read_status(pamd_ctx* c) {
    DevScalars s;
    PAMD_CU(c, cudaMemcpyAsync(&s, c->b.scal, sizeof(s), cudaMemcpyDeviceToHost, c->stream));
    PAMD_CU(c, cudaStreamSynchronize(c->stream));
    if (s.status == 0) return PAMD_OK;
    // report once, then clear so that the caller can repair the state and go on
    const int zero[2] = {0, -1};
    PAMD_CU(c, cudaMemcpyAsync(&c->b.scal->status, zero, sizeof(zero), cudaMemcpyHostToDevice, c->stream));
    PAMD_CU(c, cudaStreamSynchronize(c->stream));
    if (s.status == PAMD_ENONFINITE)
        return fail(PAMD_ENONFINITE, "non-finite energy in replica " + std::to_string(s.bad_replica));
    if (s.status == PAMD_EPOPSIZE)
        return fail(PAMD_EPOPSIZE, "resampling produced " + std::to_string(s.R_new) +
                                       " replicas (capacity " + std::to_string(c->R) + ")");
    return fail(s.status, "device status " + std::to_string(s.status));
}

int ensure_obs_cap(pamd_ctx* c, int n) {
    if (c->obs_cap >= n) return PAMD_OK;
    void* p = dalloc(c, sizeof(pamd_obs) * (size_t)n);
    if (!p) return fail(PAMD_ENOMEM, "observable buffer");
    c->b.obs = (pamd_obs*)p;  // the old buffer stays owned until destroy
    c->obs_cap = n;
    return PAMD_OK;
}

}  // namespace

namespace pamd {
cudaError_t ensure_dyn_smem(const void* fn, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    size_t& have = done[{fn, dev}];
    if (bytes <= have) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) have = bytes;
    return e;
}

void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace pamd

namespace {

// Whole batched anneal as one CUDA graph: the batched propagate launch, then
// per molecule its resampling and measurement, for every temperature step.
int anneal_batch(pamd_ctx* c, int32_t K, const double* T, int32_t theta, double dt_ps,
                 int32_t resample, pamd_obs* per_step_out) {
    if (K < 0 || !T) return fail(PAMD_EINVAL, "K must be >= 0 and T non-null");
    if (theta < 0 || !(dt_ps > 0) || !std::isfinite(dt_ps)) return fail(PAMD_EINVAL, "theta / dt");
    for (int i = 0; i <= K; ++i)
        if (!(T[i] > 0) || !std::isfinite(T[i])) return fail(PAMD_EINVAL, "temperatures must be > 0");
    int rc;
    for (pamd_ctx* sub : c->subs) {
        if ((rc = ensure_obs_cap(sub, K + 1))) return rc;
        if (sub->cur_is_alt) {
            const size_t st = state_bytes(sub);
            PAMD_CU(c, cudaMemcpyAsync(sub->b.state, sub->b.state_alt, st, cudaMemcpyDeviceToDevice, c->stream));
            PAMD_CU(c, cudaMemcpyAsync(sub->b.E, sub->b.E_alt, 8 * (size_t)sub->R, cudaMemcpyDeviceToDevice, c->stream));
            PAMD_CU(c, cudaMemcpyAsync(sub->b.fam, sub->b.fam_alt, 4 * (size_t)sub->R, cudaMemcpyDeviceToDevice, c->stream));
            sub->cur_is_alt = false;
        }
    }
    GraphKey key;
    key.K = K;
    key.theta = theta;
    key.resample = resample ? 1 : 0;
    key.dt = dt_ps;
    key.T.assign(T, T + K + 1);
    if (c->mlp) {
        // A force model issues five launches per MD step: queue the anneal
        // directly instead of capturing a graph of that size.
        PAMD_CU(c, launch_set_counters(c, c->step, c->resample_index));
        int err = launch_prop(c, theta, dt_ps, T[0], c->b.counters, 0u, nullptr);
        if (!err && launch_observe(c, T[0], c->b.obs) != cudaSuccess) err = PAMD_ECUDA;
        for (int i = 1; i <= K && !err; ++i) {
            if (launch_resample(c, T[i - 1], T[i], resample ? 1 : 0, c->b.counters, (uint32_t)i) != cudaSuccess) {
                err = PAMD_ECUDA;
                break;
            }
            c->cur_is_alt = !c->cur_is_alt;
            err = launch_prop(c, theta, dt_ps, T[i], c->b.counters, (uint32_t)i * (uint32_t)theta, nullptr);
            if (!err && launch_observe(c, T[i], c->b.obs + i) != cudaSuccess) err = PAMD_ECUDA;
        }
        if (err) {
            c->broken = true;
            return err == PAMD_ECUDA ? fail(PAMD_ECUDA, "anneal with force model: " + g_err) : err;
        }
        if (c->cur_is_alt) {
            const size_t st_bytes = state_bytes(c);
            PAMD_CU(c, cudaMemcpyAsync(c->b.state, c->b.state_alt, st_bytes, cudaMemcpyDeviceToDevice, c->stream));
            PAMD_CU(c, cudaMemcpyAsync(c->b.E, c->b.E_alt, 8 * (size_t)c->R, cudaMemcpyDeviceToDevice, c->stream));
            PAMD_CU(c, cudaMemcpyAsync(c->b.fam, c->b.fam_alt, 4 * (size_t)c->R, cudaMemcpyDeviceToDevice, c->stream));
            c->cur_is_alt = false;
        }
    } else if (!c->graph_exec || !(c->graph_key == key)) {
        if (c->graph_exec) {
            cudaGraphExecDestroy(c->graph_exec);
            c->graph_exec = nullptr;
        }
        cudaGraph_t g = nullptr;
        PAMD_CU(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        long long before = c->launches;
        for (pamd_ctx* sub : c->subs) before += sub->launches;
        int err = launch_prop_batch(c, theta, dt_ps, T[0], true, 0u);
        for (pamd_ctx* sub : c->subs)
            if (!err && launch_observe(sub, T[0], sub->b.obs) != cudaSuccess) err = PAMD_ECUDA;
        for (int i = 1; i <= K && !err; ++i) {
            for (pamd_ctx* sub : c->subs) {
                if (launch_resample(sub, T[i - 1], T[i], resample ? 1 : 0, sub->b.counters, (uint32_t)i) != cudaSuccess) {
                    err = PAMD_ECUDA;
                    break;
                }
                sub->cur_is_alt = !sub->cur_is_alt;
            }
            if (!err) err = launch_prop_batch(c, theta, dt_ps, T[i], true, (uint32_t)i * (uint32_t)theta);
            for (pamd_ctx* sub : c->subs)
                if (!err && launch_observe(sub, T[i], sub->b.obs + i) != cudaSuccess) err = PAMD_ECUDA;
        }
        for (pamd_ctx* sub : c->subs) {
            if (!err && sub->cur_is_alt) {
                const size_t st = state_bytes(sub);
                if (cudaMemcpyAsync(sub->b.state, sub->b.state_alt, st, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
                    cudaMemcpyAsync(sub->b.E, sub->b.E_alt, 8 * (size_t)sub->R, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
                    cudaMemcpyAsync(sub->b.fam, sub->b.fam_alt, 4 * (size_t)sub->R, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
                    err = PAMD_ECUDA;
            }
            sub->cur_is_alt = false;
        }
        long long after = c->launches;
        for (pamd_ctx* sub : c->subs) after += sub->launches;
        c->graph_kernels = after - before;
        // the captured launches are counted when the graph runs, not now
        c->launches -= c->graph_kernels;
        cudaError_t ec = cudaStreamEndCapture(c->stream, &g);
        if (err || ec != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            c->broken = true;
            return fail(PAMD_ECUDA, std::string("batched anneal capture failed: ") + cudaGetErrorString(ec));
        }
        cudaError_t ei = cudaGraphInstantiate(&c->graph_exec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) return cuda_fail(c, ei, "graph instantiate");
        c->graph_key = key;
    }
    for (pamd_ctx* sub : c->subs) {
        cudaError_t e = launch_set_counters(sub, sub->step, sub->resample_index);
        if (e != cudaSuccess) return cuda_fail(c, e, "set counters");
    }
    PAMD_CU(c, cudaGraphLaunch(c->graph_exec, c->stream));
    c->launches += c->graph_kernels;
    for (pamd_ctx* sub : c->subs) {
        sub->step += (uint32_t)(K + 1) * (uint32_t)theta;
        sub->resample_index += (uint32_t)K;
    }
    const int M = (int)c->subs.size();
    std::vector<pamd_obs> tmp((size_t)(K + 1));
    for (int m = 0; m < M; ++m) {
        pamd_ctx* sub = c->subs[m];
        if (per_step_out) {
            PAMD_CU(c, cudaMemcpyAsync(tmp.data(), sub->b.obs, sizeof(pamd_obs) * (size_t)(K + 1),
                                       cudaMemcpyDeviceToHost, c->stream));
            PAMD_CU(c, cudaStreamSynchronize(c->stream));
            for (int i = 0; i <= K; ++i) {
                per_step_out[(size_t)i * M + m] = tmp[i];
                per_step_out[(size_t)i * M + m].pad_ = 0;
            }
        }
        if ((rc = read_status(sub))) return rc;
    }
    return PAMD_OK;
}

}  // namespace

extern "C" {

void pamd_options_default(pamd_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->gamma_per_ps = 1.0;
    o->precision = PAMD_PREC_MIXED;
}

const char* pamd_last_error(void) { return g_err.c_str(); }

int pamd_init(pamd_ctx** out, const pamd_topology* top, int64_t R, double T0, uint64_t seed,
              const pamd_options* opt) {
    g_err.clear();
    if (!out || !top) return fail(PAMD_EINVAL, "null argument");
    *out = nullptr;
    if (R < 1 || R > 0x7fffffffLL) return fail(PAMD_EINVAL, "R must be in 1 .. 2^31-1");
    if (!(T0 > 0) || !std::isfinite(T0)) return fail(PAMD_EINVAL, "T0 must be > 0");
    pamd_options o;
    pamd_options_default(&o);
    if (opt) o = *opt;
    if (!(o.gamma_per_ps >= 0) || !std::isfinite(o.gamma_per_ps))
        return fail(PAMD_EINVAL, "gamma must be >= 0");
    if (o.precision != PAMD_PREC_MIXED && o.precision != PAMD_PREC_FP64)
        return fail(PAMD_EUNSUPPORTED, "precision must be PAMD_PREC_MIXED or PAMD_PREC_FP64");
    if (o.warps_per_block < 0 || o.warps_per_block > 8)
        return fail(PAMD_EINVAL, "warps_per_block must be 0..8");
    if (o.mol_id < 0 || o.mol_id > 0xffffff) return fail(PAMD_EINVAL, "mol_id must be 0..2^24-1");
    if (o.replicas_per_lane < 0 || o.replicas_per_lane > 2)
        return fail(PAMD_EINVAL, "replicas_per_lane must be 0, 1 or 2");
    if (o.pair_arith < PAMD_PAIRS_AUTO || o.pair_arith > PAMD_PAIRS_PACKED)
        return fail(PAMD_EINVAL, "pair_arith must be PAMD_PAIRS_AUTO, _SCALAR or _PACKED");
    if (o.pair_arith == PAMD_PAIRS_PACKED && o.replicas_per_lane == 2)
        return fail(PAMD_EINVAL, "packed pair arithmetic runs one replica per lane group");
    if ((o.dev_alloc == nullptr) != (o.dev_free == nullptr))
        return fail(PAMD_EINVAL, "dev_alloc and dev_free must both be set or both be NULL");
    if (o.resample_rule < PAMD_RESAMPLE_MULTINOMIAL || o.resample_rule > PAMD_RESAMPLE_POISSON)
        return fail(PAMD_EINVAL, "resample_rule must be one of the PAMD_RESAMPLE_* rules");
    // rules whose copy numbers change the population size: a fixed capacity
    // of slots, the live size on the device
    const bool variable = o.resample_rule == PAMD_RESAMPLE_NEAREST || o.resample_rule == PAMD_RESAMPLE_POISSON;
    long long capacity = R;
    if (variable) {
        if (o.precision != PAMD_PREC_MIXED || o.replicas_per_lane == 2)
            return fail(PAMD_EUNSUPPORTED, "variable population sizes need mixed precision and one replica per lane group");
        capacity = R + 8 * (long long)std::ceil(std::sqrt((double)R)) + 64;
        if (capacity > 0x7fffffffLL) return fail(PAMD_EINVAL, "R too large for a variable population");
    }

    pamd_ctx* c = new (std::nothrow) pamd_ctx();
    if (!c) return fail(PAMD_ENOMEM, "host allocation");
    c->R = capacity;
    c->R_target = R;
    c->variable = variable;
    c->resample_rule = o.resample_rule;
    c->precision = o.precision;
    c->gamma = o.gamma_per_ps;
    c->seed = seed;
    c->mol = o.mol_id;
    c->dev_alloc = o.dev_alloc;
    c->dev_free = o.dev_free;
    c->alloc_user = o.alloc_user;
    std::vector<unsigned char> blob;
    TopoLayout lay0;
    int rc = build_topology(top, o.lanes_per_replica, &lay0, blob);
    if (rc) {
        delete c;
        return rc;
    }
    c->host_top.assign(top);
    c->lanes_req = o.lanes_per_replica;
    c->pair_arith = o.pair_arith;
    c->N = lay0.n_atoms;
    c->Np = lay0.n_pad;
    auto bail = [&](int code, const std::string& m) {
        free_all(c);
        if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
        delete c;
        return fail(code, m);
    };
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return bail(PAMD_ECUDA, "no CUDA device");
    if (o.stream) {
        c->stream = (cudaStream_t)o.stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(PAMD_ECUDA, "stream creation");
        c->own_stream = true;
    }
    // launch shape
    int variant = kVarScalar;
    if (o.replicas_per_lane == 2)
        variant = kVarPaired;
    else if (o.pair_arith == PAMD_PAIRS_PACKED)
        variant = kVarPacked;
    else if (o.pair_arith == PAMD_PAIRS_AUTO && o.precision == PAMD_PREC_MIXED && packed_ok(lay0))
        variant = kVarPacked;  // the faster arithmetic wherever its layout applies
    if ((rc = set_launch_shape(c, lay0, o.warps_per_block, variant))) {
        const std::string m = g_err;
        return bail(rc, m);
    }

    // host-side tables
    c->host_mass.assign(top->mass, top->mass + c->N);
    std::vector<float> masses(c->Np, 0.0f), x0(3 * (size_t)c->Np, 0.0f);
    double com[3] = {0, 0, 0}, mt = 0;
    for (int i = 0; i < c->N; ++i) {
        for (int q = 0; q < 3; ++q) com[q] += top->mass[i] * top->x0[3 * i + q];
        mt += top->mass[i];
    }
    for (int i = 0; i < c->N; ++i) {
        masses[i] = (float)top->mass[i];
        for (int q = 0; q < 3; ++q) x0[(size_t)q * c->Np + i] = (float)(top->x0[3 * i + q] - com[q] / mt);
    }
    // buffers
    const size_t st_bytes = state_bytes(c);
    c->n_blk = (int)((c->R + 1023) / 1024);  // R here: the slots (capacity)
    Buffers& b = c->b;
    b.state = (float*)dalloc(c, st_bytes);
    b.state_alt = (float*)dalloc(c, st_bytes);
    b.E = (double*)dalloc(c, sizeof(double) * c->R);
    b.E_alt = (double*)dalloc(c, sizeof(double) * c->R);
    b.fam = (int32_t*)dalloc(c, sizeof(int32_t) * c->R);
    b.fam_alt = (int32_t*)dalloc(c, sizeof(int32_t) * c->R);
    b.ke = (double*)dalloc(c, sizeof(double) * c->R);
    b.rg = (double*)dalloc(c, sizeof(double) * c->R);
    b.masses = (float*)dalloc(c, sizeof(float) * c->Np);
    b.topo = (unsigned char*)dalloc(c, blob.size());
    c->topo_cap = blob.size();
    b.x0 = (float*)dalloc(c, sizeof(float) * 3 * c->Np);
    b.W = (unsigned long long*)dalloc(c, 8 * (size_t)c->R);
    b.C = (unsigned long long*)dalloc(c, 8 * (size_t)c->R);
    b.cnt = (int32_t*)dalloc(c, 4 * (size_t)c->R);
    b.cnt_incl = (int32_t*)dalloc(c, 4 * (size_t)c->R);
    b.blk_u64 = (unsigned long long*)dalloc(c, 8 * (size_t)c->n_blk);
    b.blk_f64 = (double*)dalloc(c, 8 * (size_t)c->n_blk);
    b.blk_i32 = (int32_t*)dalloc(c, 8 * (size_t)c->n_blk);
    b.flags = (unsigned char*)dalloc(c, (size_t)c->R);
    b.obs_part = (double*)dalloc(c, sizeof(double) * (64 * 5 + 1) * (size_t)c->n_blk);
    b.scal = (DevScalars*)dalloc(c, sizeof(DevScalars));
    b.counters = (uint32_t*)dalloc(c, 16);
    if (!b.state || !b.state_alt || !b.E || !b.E_alt || !b.fam || !b.fam_alt || !b.ke || !b.rg ||
        !b.masses || !b.topo || !b.x0 || !b.W || !b.C || !b.cnt || !b.cnt_incl || !b.blk_u64 ||
        !b.blk_f64 || !b.blk_i32 || !b.flags || !b.obs_part || !b.scal || !b.counters)
        return bail(PAMD_ENOMEM, "device allocation failed");
    if (ensure_obs_cap(c, 2)) return bail(PAMD_ENOMEM, "device allocation failed");
    std::vector<unsigned char> t64;
    if (is_f64(c)) {
        if ((rc = build_topo_f64(c, top, t64))) {
            const std::string m = g_err;
            return bail(rc, m);
        }
    }
    bool ok = cudaMemcpyAsync(b.masses, masses.data(), sizeof(float) * c->Np, cudaMemcpyHostToDevice, c->stream) == cudaSuccess &&
              cudaMemcpyAsync(b.topo, blob.data(), blob.size(), cudaMemcpyHostToDevice, c->stream) == cudaSuccess &&
              cudaMemcpyAsync(b.x0, x0.data(), sizeof(float) * 3 * c->Np, cudaMemcpyHostToDevice, c->stream) == cudaSuccess &&
              cudaMemsetAsync(b.state_alt, 0, st_bytes, c->stream) == cudaSuccess &&
              cudaMemsetAsync(b.ke, 0, sizeof(double) * c->R, c->stream) == cudaSuccess &&
              cudaMemsetAsync(b.rg, 0, sizeof(double) * c->R, c->stream) == cudaSuccess &&
              (t64.empty() || cudaMemcpyAsync(c->top64_blob, t64.data(), t64.size(),
                                              cudaMemcpyHostToDevice, c->stream) == cudaSuccess) &&
              launch_init(c, T0) == cudaSuccess &&
              launch_set_counters(c, 0, 0) == cudaSuccess &&
              cudaStreamSynchronize(c->stream) == cudaSuccess;
    if (!ok) return bail(PAMD_ECUDA, std::string("initialisation: ") + cudaGetErrorString(cudaGetLastError()));
    if (o.autotune) {
        const int r = pamd_autotune(c, 20, nullptr);
        if (r) {
            const std::string m = g_err;
            return bail(r, "autotune: " + m);
        }
    }
    *out = c;
    return PAMD_OK;
}

int pamd_init_batch(pamd_ctx** out, int32_t n_mol, const pamd_topology* tops, const int64_t* R,
                    const double* T0, uint64_t seed, const pamd_options* opt) {
    g_err.clear();
    if (!out || !tops || !R || !T0) return fail(PAMD_EINVAL, "null argument");
    *out = nullptr;
    if (n_mol < 1 || n_mol > kMaxBatchMols) return fail(PAMD_EINVAL, "n_mol must be 1..64");
    pamd_options o;
    pamd_options_default(&o);
    if (opt) o = *opt;
    if (o.precision != PAMD_PREC_MIXED)
        return fail(PAMD_EUNSUPPORTED, "the batched kernel runs the mixed-precision path only");
    if (o.replicas_per_lane > 1) return fail(PAMD_EUNSUPPORTED, "the batched kernel runs one replica per lane group");
    if (o.resample_rule == PAMD_RESAMPLE_NEAREST || o.resample_rule == PAMD_RESAMPLE_POISSON)
        return fail(PAMD_EUNSUPPORTED, "batched anneals keep a fixed population size");
    if ((o.dev_alloc == nullptr) != (o.dev_free == nullptr))
        return fail(PAMD_EINVAL, "dev_alloc and dev_free must both be set or both be NULL");
    for (int m = 0; m < n_mol; ++m)
        if (R[m] < 1 || R[m] > 0x7fffffffLL) return fail(PAMD_EINVAL, "every R must be in 1 .. 2^31-1");
    pamd_ctx* c = new (std::nothrow) pamd_ctx();
    if (!c) return fail(PAMD_ENOMEM, "host allocation");
    c->dev_alloc = o.dev_alloc;
    c->dev_free = o.dev_free;
    c->alloc_user = o.alloc_user;
    c->seed = seed;
    auto bail = [&](int code, const std::string& m) {
        for (pamd_ctx* s : c->subs) pamd_destroy(s);
        c->subs.clear();
        for (cudaStream_t gs : c->group_streams) cudaStreamDestroy(gs);
        for (cudaEvent_t ge : c->group_events) cudaEventDestroy(ge);
        if (c->fork_event) cudaEventDestroy(c->fork_event);
        free_all(c);
        if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
        delete c;
        return fail(code, m);
    };
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return bail(PAMD_ECUDA, "no CUDA device");
    if (o.stream) {
        c->stream = (cudaStream_t)o.stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(PAMD_ECUDA, "stream creation");
        c->own_stream = true;
    }
    // one ordinary context per molecule, sharing the stream
    std::vector<std::pair<int, int>> order;  // (N, m)
    for (int m = 0; m < n_mol; ++m) {
        pamd_options so = o;
        so.mol_id = m;
        so.stream = c->stream;
        so.warps_per_block = kBatchThreads / 32;
        so.autotune = 0;
        so.replicas_per_lane = 1;
        so.lanes_per_replica = tops[m].n_atoms >= 1 && tops[m].n_atoms <= PAMD_MAX_ATOMS
                                   ? batch_lanes(tops[m].n_atoms) : 0;
        // the packed pair arithmetic wherever its chain layout applies,
        // unless the caller asked for the scalar one
        const bool try_packed = o.pair_arith != PAMD_PAIRS_SCALAR && is_linear_chain(&tops[m]);
        so.pair_arith = try_packed ? PAMD_PAIRS_PACKED : PAMD_PAIRS_SCALAR;
        pamd_ctx* sub = nullptr;
        int rc = pamd_init(&sub, &tops[m], R[m], T0[m], seed, &so);
        if (rc == PAMD_EUNSUPPORTED && try_packed) {
            so.pair_arith = PAMD_PAIRS_SCALAR;
            rc = pamd_init(&sub, &tops[m], R[m], T0[m], seed, &so);
        }
        if (rc) {
            const std::string msg = "molecule " + std::to_string(m) + ": " + g_err;
            return bail(rc, msg);
        }
        c->subs.push_back(sub);
        if (o.autotune && sub->N >= 3) {
            // measured choice among the batched kernel's shapes
            const int trc = autotune_with(sub, 20, TuneLimits{3, 7, false, sub->pair_arith == PAMD_PAIRS_PACKED,
                                                                  {kBatchThreads / 32}, -2}, nullptr);
            if (trc && trc != PAMD_EUNSUPPORTED) {
                const std::string msg = "molecule " + std::to_string(m) + ": " + g_err;
                return bail(trc, msg);
            }
        }
        if (sub->warps_per_block != kBatchThreads / 32 || sub->lay.per_lane < 3 || sub->lay.per_lane > 7)
            return bail(PAMD_EUNSUPPORTED, "molecule " + std::to_string(m) + " does not fit the batched kernel");
        c->R += R[m];
        c->N = std::max(c->N, sub->N);
        order.push_back({sub->N, m});
    }
    // work lists: molecules grouped by atoms per lane and pair arithmetic
    // (one launch per group, largest total work first), by decreasing size
    // within a group, each cut into one CTA's worth of replicas
    std::stable_sort(order.begin(), order.end(), [](auto a, auto b) { return a.first > b.first; });
    std::vector<int4> items;
    std::vector<std::pair<double, pamd_ctx::BatchGroup>> groups;
    for (int gk = 0; gk < 10; ++gk) {
        const int Bg = 3 + gk / 2;
        const bool packed = (gk & 1) != 0;
        pamd_ctx::BatchGroup gr{Bg, (int)items.size(), 0, 0, 0, packed};
        double work = 0.0;
        for (auto& om : order) {
            pamd_ctx* sub = c->subs[om.second];
            if (sub->lay.per_lane != Bg || (sub->lay.packed != 0) != packed) continue;
            for (long long k0 = 0; k0 < sub->R; k0 += sub->rpb)
                items.push_back(make_int4(om.second, (int)k0, (int)std::min<long long>(k0 + sub->rpb, sub->R), 0));
            gr.smem = std::max(gr.smem, prop_smem(sub));
            work += (double)sub->R * sub->N * sub->N;
        }
        gr.n_items = (int)items.size() - gr.first_item;
        if (gr.n_items == 0) continue;
        int occ = 0;
        const cudaError_t e = packed ? propagate_batch_x2_occupancy(Bg, gr.smem, &occ)
                                     : propagate_batch_occupancy(Bg, gr.smem, &occ);
        if (e != cudaSuccess || occ < 1)
            return bail(PAMD_ECUDA, std::string("batched kernel occupancy: ") + cudaGetErrorString(e));
        gr.grid = std::min(gr.n_items, c->num_sms * occ);
        groups.push_back({work, gr});
    }
    std::stable_sort(groups.begin(), groups.end(), [](auto a, auto b) { return a.first > b.first; });
    for (auto& wg : groups) c->groups.push_back(wg.second);
    // one stream and completion event per group, forked from the context's stream
    if (c->groups.size() > 1) {
        if (cudaEventCreateWithFlags(&c->fork_event, cudaEventDisableTiming) != cudaSuccess)
            return bail(PAMD_ECUDA, "group streams");
        for (size_t q = 0; q < c->groups.size(); ++q) {
            cudaStream_t gs = nullptr;
            cudaEvent_t ge = nullptr;
            if (cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking) != cudaSuccess)
                return bail(PAMD_ECUDA, "group streams");
            c->group_streams.push_back(gs);
            if (cudaEventCreateWithFlags(&ge, cudaEventDisableTiming) != cudaSuccess)
                return bail(PAMD_ECUDA, "group streams");
            c->group_events.push_back(ge);
        }
    }
    c->n_items = (int)items.size();
    c->items = (int4*)dalloc(c, sizeof(int4) * items.size());
    c->queue = (int*)dalloc(c, sizeof(int) * c->groups.size());
    if (!c->items || !c->queue) return bail(PAMD_ENOMEM, "work list");
    if (cudaMemcpyAsync(c->items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice,
                        c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return bail(PAMD_ECUDA, "work list upload");
    *out = c;
    return PAMD_OK;
}

int32_t pamd_batch_size(pamd_ctx* c) { return c ? (int32_t)c->subs.size() : -1; }

pamd_ctx* pamd_batch_sub(pamd_ctx* c, int32_t m) {
    if (!c || m < 0 || m >= (int32_t)c->subs.size()) {
        g_err = "no such molecule in this batch";
        return nullptr;
    }
    return c->subs[m];
}

int pamd_reset(pamd_ctx* c, double T0, uint64_t seed) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (is_batch(c)) {
        for (pamd_ctx* sub : c->subs)
            if ((rc = pamd_reset(sub, T0, seed))) return rc;
        return PAMD_OK;
    }
    if (!(T0 > 0) || !std::isfinite(T0)) return fail(PAMD_EINVAL, "T0 must be > 0");
    c->seed = seed;
    c->cur_is_alt = false;
    c->step = 0;
    c->resample_index = 0;
    cudaError_t e = launch_init(c, T0);
    if (e != cudaSuccess) return cuda_fail(c, e, "reset");
    return PAMD_OK;
}

int pamd_propagate(pamd_ctx* c, int32_t theta, double dt_ps, double T) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (is_batch(c)) {
        if (theta < 0 || !(dt_ps > 0) || !(T > 0) || !std::isfinite(dt_ps) || !std::isfinite(T))
            return fail(PAMD_EINVAL, "theta >= 0, dt > 0 and T > 0 required");
        if ((rc = launch_prop_batch(c, theta, dt_ps, T, false, 0))) return rc;
        for (pamd_ctx* sub : c->subs) sub->step += (uint32_t)theta;
        return PAMD_OK;
    }
    if (theta < 0) return fail(PAMD_EINVAL, "theta must be >= 0");
    if (!(dt_ps > 0) || !std::isfinite(dt_ps)) return fail(PAMD_EINVAL, "dt must be > 0");
    if (!(T > 0) || !std::isfinite(T)) return fail(PAMD_EINVAL, "T must be > 0");
    rc = launch_prop(c, theta, dt_ps, T, nullptr, c->step, nullptr);
    if (rc) return rc;
    c->step += (uint32_t)theta;
    return PAMD_OK;
}

int pamd_resample(pamd_ctx* c, double T_prev, double T_next, int32_t* copies_out, double* lnQ_out) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (is_batch(c)) {
        if (!(T_prev > 0) || !(T_next > 0) || !std::isfinite(T_prev) || !std::isfinite(T_next))
            return fail(PAMD_EINVAL, "temperatures must be > 0");
        long long off = 0;
        for (size_t m = 0; m < c->subs.size(); ++m) {
            pamd_ctx* sub = c->subs[m];
            if ((rc = pamd_resample(sub, T_prev, T_next, copies_out ? copies_out + off : nullptr,
                                    lnQ_out ? lnQ_out + m : nullptr)))
                return rc;
            off += sub->R;
        }
        return PAMD_OK;
    }
    if (!(T_prev > 0) || !(T_next > 0) || !std::isfinite(T_prev) || !std::isfinite(T_next))
        return fail(PAMD_EINVAL, "temperatures must be > 0");
    c->resample_index += 1;
    cudaError_t e = launch_resample(c, T_prev, T_next, 1, nullptr, c->resample_index);
    if (e != cudaSuccess) return cuda_fail(c, e, "resample launch");
    c->cur_is_alt = !c->cur_is_alt;
    if (copies_out)
        PAMD_CU(c, cudaMemcpyAsync(copies_out, c->b.cnt, sizeof(int32_t) * c->R, cudaMemcpyDeviceToHost, c->stream));
    if (lnQ_out)
        PAMD_CU(c, cudaMemcpyAsync(lnQ_out, &c->b.scal->lnQ, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (copies_out || lnQ_out) return read_status(c);
    return PAMD_OK;
}

int pamd_observables(pamd_ctx* c, double T, pamd_obs* out) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (is_batch(c)) {
        if (!out) return fail(PAMD_EINVAL, "null output");
        for (size_t m = 0; m < c->subs.size(); ++m)
            if ((rc = pamd_observables(c->subs[m], T, out + m))) return rc;
        return PAMD_OK;
    }
    if (!out) return fail(PAMD_EINVAL, "null output");
    cudaError_t e = launch_observe(c, T, c->b.obs);
    if (e != cudaSuccess) return cuda_fail(c, e, "observables launch");
    PAMD_CU(c, cudaMemcpyAsync(out, c->b.obs, sizeof(pamd_obs), cudaMemcpyDeviceToHost, c->stream));
    rc = read_status(c);
    out->pad_ = 0;
    return rc;
}

namespace {
// Row i of the energy record (pamd_record_energies) <- the current energies.
cudaError_t record_energies(pamd_ctx* c, int i) {
    if (!c->rec_E || i >= c->rec_rows) return cudaSuccess;
    return cudaMemcpyAsync(c->rec_E + (size_t)i * (size_t)c->R, cur_E(c), sizeof(double) * (size_t)c->R,
                           cudaMemcpyDeviceToDevice, c->stream);
}
}  // namespace

int pamd_record_energies(pamd_ctx* c, double* E_dev, int32_t rows) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (c->variable) return fail(PAMD_EUNSUPPORTED, "not available with a variable population size");
    if (is_batch(c)) return fail(PAMD_EINVAL, "energy recording: single-molecule contexts only");
    if (rows < 0 || (rows > 0 && !E_dev)) return fail(PAMD_EINVAL, "energy recording: rows >= 0, E_dev for rows > 0");
    c->rec_E = rows > 0 ? E_dev : nullptr;
    c->rec_rows = rows > 0 ? rows : 0;
    return PAMD_OK;
}

int pamd_next_temperature(pamd_ctx* c, double T_prev, double T_final, double alpha_target,
                          double* T_next_out, double* alpha_out) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (c->variable) return fail(PAMD_EUNSUPPORTED, "not available with a variable population size");
    if (is_batch(c)) return fail(PAMD_EINVAL, "overlap step: single-molecule contexts only");
    if (!T_next_out) return fail(PAMD_EINVAL, "overlap step: T_next_out is required");
    if ((rc = overlap_check_args(c->R, T_prev, T_final, alpha_target))) return rc;
    if (!c->ov_work) {
        c->ov_work = dalloc(c, overlap_work_bytes(c->R));
        if (!c->ov_work) return fail(PAMD_ENOMEM, "overlap step scratch");
    }
    rc = overlap_step(c->stream, cur_E(c), c->R, T_prev, T_final, alpha_target, c->ov_work, c->num_sms,
                      T_next_out, alpha_out, &c->launches);
    if (rc == PAMD_ECUDA) c->broken = true;
    return rc;
}

int pamd_anneal_adaptive(pamd_ctx* c, double T0, double T_final, double alpha_target, int32_t theta,
                         double dt_ps, int32_t max_steps, int32_t resample, pamd_obs* obs_out,
                         double* T_out, int32_t* n_temps_out) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (c->variable) return fail(PAMD_EUNSUPPORTED, "not available with a variable population size");
    if (is_batch(c)) return fail(PAMD_EINVAL, "adaptive anneal: single-molecule contexts only");
    if (!(T0 > 0) || !std::isfinite(T0) || !(T_final > 0) || !(T_final < T0))
        return fail(PAMD_EINVAL, "adaptive anneal: 0 < T_final < T0 required");
    if (!(alpha_target > 0) || !(alpha_target < 1))
        return fail(PAMD_EINVAL, "adaptive anneal: alpha_target must be in (0, 1)");
    if (max_steps < 0 || theta < 0 || !(dt_ps > 0) || !std::isfinite(dt_ps))
        return fail(PAMD_EINVAL, "adaptive anneal: max_steps >= 0, theta >= 0, dt > 0");
    pamd_obs o;
    if ((rc = pamd_propagate(c, theta, dt_ps, T0)) || (rc = pamd_observables(c, T0, &o))) return rc;
    PAMD_CU(c, record_energies(c, 0));
    if (obs_out) obs_out[0] = o;
    if (T_out) T_out[0] = T0;
    int n = 1;
    double T = T0;
    for (int i = 1; i <= max_steps && T > T_final; ++i) {
        double Tn = T;
        if ((rc = pamd_next_temperature(c, T, T_final, alpha_target, &Tn, nullptr))) return rc;
        if (!(Tn < T))
            return fail(PAMD_EINVAL, "adaptive anneal: no lower temperature meets the overlap target "
                                     "(alpha_target too close to 1 for this population)");
        c->resample_index += 1;
        cudaError_t e = launch_resample(c, T, Tn, resample ? 1 : 0, nullptr, c->resample_index);
        if (e != cudaSuccess) return cuda_fail(c, e, "resample launch");
        c->cur_is_alt = !c->cur_is_alt;
        if ((rc = pamd_propagate(c, theta, dt_ps, Tn)) || (rc = pamd_observables(c, Tn, &o))) return rc;
        PAMD_CU(c, record_energies(c, i));
        if (obs_out) obs_out[i] = o;
        if (T_out) T_out[i] = Tn;
        T = Tn;
        ++n;
    }
    if (n_temps_out) *n_temps_out = n;
    return read_status(c);
}

int pamd_anneal(pamd_ctx* c, int32_t K, const double* T, int32_t theta, double dt_ps,
                int32_t resample, pamd_obs* per_step_out) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (is_batch(c)) return anneal_batch(c, K, T, theta, dt_ps, resample, per_step_out);
    if (K < 0 || !T) return fail(PAMD_EINVAL, "K must be >= 0 and T non-null");
    if (theta < 0 || !(dt_ps > 0) || !std::isfinite(dt_ps)) return fail(PAMD_EINVAL, "theta / dt");
    for (int i = 0; i <= K; ++i)
        if (!(T[i] > 0) || !std::isfinite(T[i])) return fail(PAMD_EINVAL, "temperatures must be > 0");
    if ((rc = ensure_obs_cap(c, K + 1))) return rc;
    GraphKey key;
    key.K = K;
    key.theta = theta;
    key.resample = resample ? 1 : 0;
    key.dt = dt_ps;
    key.T.assign(T, T + K + 1);
    key.rec = c->rec_E;
    key.rec_rows = c->rec_rows;
    // the captured graph starts from the main buffers
    if (c->cur_is_alt) {
        const size_t st_bytes = state_bytes(c);
        PAMD_CU(c, cudaMemcpyAsync(c->b.state, c->b.state_alt, st_bytes, cudaMemcpyDeviceToDevice, c->stream));
        PAMD_CU(c, cudaMemcpyAsync(c->b.E, c->b.E_alt, 8 * (size_t)c->R, cudaMemcpyDeviceToDevice, c->stream));
        PAMD_CU(c, cudaMemcpyAsync(c->b.fam, c->b.fam_alt, 4 * (size_t)c->R, cudaMemcpyDeviceToDevice, c->stream));
        c->cur_is_alt = false;
    }
    if (c->mlp) {
        // With a force model each temperature's theta MD steps are one WHILE
        // node of the graph (step kernel and four GEMMs per iteration).  The
        // graph holds the model's workspace pointers and energy scale.
        if (c->mlp->broken) return fail(PAMD_ESTATE, "force model unusable after an earlier CUDA error");
        if ((rc = mlp_prepare_capture(c->mlp))) return rc;
        key.model = c->mlp;
        key.model_gen = c->mlp->work_gen;
        key.mu_E = c->mlp->mu_E;
        key.sigma_E = c->mlp->sigma_E;
    }
    if (!c->graph_exec || !(c->graph_key == key)) {
        if (c->graph_exec) {
            cudaGraphExecDestroy(c->graph_exec);
            c->graph_exec = nullptr;
        }
        cudaGraph_t g = nullptr;
        PAMD_CU(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        const long long before = c->launches;
        int err = launch_prop(c, theta, dt_ps, T[0], c->b.counters, 0u, nullptr);
        if (!err && launch_observe(c, T[0], c->b.obs) != cudaSuccess) err = PAMD_ECUDA;
        if (!err && record_energies(c, 0) != cudaSuccess) err = PAMD_ECUDA;
        for (int i = 1; i <= K && !err; ++i) {
            if (launch_resample(c, T[i - 1], T[i], resample ? 1 : 0, c->b.counters, (uint32_t)i) != cudaSuccess) {
                err = PAMD_ECUDA;
                break;
            }
            c->cur_is_alt = !c->cur_is_alt;
            err = launch_prop(c, theta, dt_ps, T[i], c->b.counters, (uint32_t)i * (uint32_t)theta, nullptr);
            if (!err && launch_observe(c, T[i], c->b.obs + i) != cudaSuccess) err = PAMD_ECUDA;
            if (!err && record_energies(c, i) != cudaSuccess) err = PAMD_ECUDA;
        }
        if (!err && c->cur_is_alt) {
            const size_t st_bytes = state_bytes(c);
            if (cudaMemcpyAsync(c->b.state, c->b.state_alt, st_bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
                cudaMemcpyAsync(c->b.E, c->b.E_alt, 8 * (size_t)c->R, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
                cudaMemcpyAsync(c->b.fam, c->b.fam_alt, 4 * (size_t)c->R, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
                err = PAMD_ECUDA;
        }
        c->cur_is_alt = false;
        c->graph_kernels = c->launches - before;
        c->launches = before;
        cudaError_t ec = cudaStreamEndCapture(c->stream, &g);
        if (err || ec != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            c->broken = true;
            return fail(PAMD_ECUDA, std::string("anneal capture failed: ") + cudaGetErrorString(ec) + " " + g_err);
        }
        cudaError_t ei = cudaGraphInstantiate(&c->graph_exec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) return cuda_fail(c, ei, "graph instantiate");
        c->graph_key = key;
    }
    {
        cudaError_t e = launch_set_counters(c, c->step, c->resample_index);
        if (e != cudaSuccess) return cuda_fail(c, e, "set counters");
        PAMD_CU(c, cudaGraphLaunch(c->graph_exec, c->stream));
        c->launches += c->graph_kernels;
    }
    c->step += (uint32_t)(K + 1) * (uint32_t)theta;
    c->resample_index += (uint32_t)K;
    if (per_step_out) {
        PAMD_CU(c, cudaMemcpyAsync(per_step_out, c->b.obs, sizeof(pamd_obs) * (size_t)(K + 1),
                                   cudaMemcpyDeviceToHost, c->stream));
        rc = read_status(c);
        for (int i = 0; i <= K; ++i) per_step_out[i].pad_ = 0;
        return rc;
    }
    return read_status(c);
}

int pamd_get_state(pamd_ctx* c, double* x, double* v, double* E, int32_t* fam) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (is_batch(c)) return fail(PAMD_EINVAL, "batch context: call this on pamd_batch_sub(ctx, m)");
    const int N = c->N, Np = c->Np;
    const long long R = c->R;
    std::vector<float> st;
    std::vector<double> st64;
    if ((x || v) && is_f64(c)) {
        st64.resize((size_t)R * 6 * Np);
        PAMD_CU(c, cudaMemcpyAsync(st64.data(), cur_state(c), st64.size() * 8, cudaMemcpyDeviceToHost, c->stream));
    } else if (x || v) {
        st.resize((size_t)R * 6 * Np);
        PAMD_CU(c, cudaMemcpyAsync(st.data(), cur_state(c), st.size() * 4, cudaMemcpyDeviceToHost, c->stream));
    }
    if (E) PAMD_CU(c, cudaMemcpyAsync(E, cur_E(c), 8 * (size_t)R, cudaMemcpyDeviceToHost, c->stream));
    if (fam) PAMD_CU(c, cudaMemcpyAsync(fam, cur_fam(c), 4 * (size_t)R, cudaMemcpyDeviceToHost, c->stream));
    PAMD_CU(c, cudaStreamSynchronize(c->stream));
    for (long long k = 0; k < R && (x || v); ++k) {
        for (int i = 0; i < N; ++i)
            for (int q = 0; q < 3; ++q) {
                const size_t ix = (size_t)k * 6 * Np + (size_t)q * Np + i;
                const size_t iv = ix + 3 * (size_t)Np;
                if (x) x[((size_t)k * N + i) * 3 + q] = st64.empty() ? (double)st[ix] : st64[ix];
                if (v) v[((size_t)k * N + i) * 3 + q] = st64.empty() ? (double)st[iv] : st64[iv];
            }
    }
    return PAMD_OK;
}

int pamd_set_state(pamd_ctx* c, const double* x, const double* v, const double* E, const int32_t* fam) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (is_batch(c)) return fail(PAMD_EINVAL, "batch context: call this on pamd_batch_sub(ctx, m)");
    if (!x || !v) return fail(PAMD_EINVAL, "x and v are required");
    const int N = c->N, Np = c->Np;
    const long long R = c->R;
    if (!finite_all(x, (int)std::min<long long>(R * N * 3, 0x7fffffff)) ||
        !finite_all(v, (int)std::min<long long>(R * N * 3, 0x7fffffff)))
        return fail(PAMD_EINVAL, "non-finite state");
    if (is_f64(c)) {
        std::vector<double> st((size_t)R * 6 * Np, 0.0);
        for (long long k = 0; k < R; ++k) {
            double* s = st.data() + (size_t)k * 6 * Np;
            for (int i = 0; i < N; ++i)
                for (int q = 0; q < 3; ++q) {
                    s[(size_t)q * Np + i] = x[((size_t)k * N + i) * 3 + q];
                    s[(size_t)(3 + q) * Np + i] = v[((size_t)k * N + i) * 3 + q];
                }
        }
        PAMD_CU(c, cudaMemcpyAsync(cur_state(c), st.data(), st.size() * 8, cudaMemcpyHostToDevice, c->stream));
        PAMD_CU(c, cudaStreamSynchronize(c->stream));
    } else {
        std::vector<float> st((size_t)R * 6 * Np, 0.0f);
        for (long long k = 0; k < R; ++k) {
            float* s = st.data() + (size_t)k * 6 * Np;
            for (int i = 0; i < N; ++i)
                for (int q = 0; q < 3; ++q) {
                    s[(size_t)q * Np + i] = (float)x[((size_t)k * N + i) * 3 + q];
                    s[(size_t)(3 + q) * Np + i] = (float)v[((size_t)k * N + i) * 3 + q];
                }
        }
        PAMD_CU(c, cudaMemcpyAsync(cur_state(c), st.data(), st.size() * 4, cudaMemcpyHostToDevice, c->stream));
        PAMD_CU(c, cudaStreamSynchronize(c->stream));
    }
    if (E) PAMD_CU(c, cudaMemcpyAsync(cur_E(c), E, 8 * (size_t)R, cudaMemcpyHostToDevice, c->stream));
    if (fam) PAMD_CU(c, cudaMemcpyAsync(cur_fam(c), fam, 4 * (size_t)R, cudaMemcpyHostToDevice, c->stream));
    PAMD_CU(c, cudaStreamSynchronize(c->stream));
    return PAMD_OK;
}

int pamd_forces(pamd_ctx* c, double* f, double* E) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (is_batch(c)) return fail(PAMD_EINVAL, "batch context: call this on pamd_batch_sub(ctx, m)");
    const int N = c->N, Np = c->Np;
    const long long R = c->R;
    const size_t es = is_f64(c) ? 8 : 4;
    if (!c->b.fout) {
        c->b.fout = (float*)dalloc(c, es * 3 * (size_t)Np * (size_t)R);
        if (!c->b.fout) return fail(PAMD_ENOMEM, "force buffer");
    }
    if ((rc = launch_prop(c, 0, 0.001, 300.0, nullptr, c->step, c->b.fout))) return rc;
    std::vector<float> fo;
    std::vector<double> fo64;
    if (f && is_f64(c)) {
        fo64.resize((size_t)R * 3 * Np);
        PAMD_CU(c, cudaMemcpyAsync(fo64.data(), c->b.fout, fo64.size() * 8, cudaMemcpyDeviceToHost, c->stream));
    } else if (f) {
        fo.resize((size_t)R * 3 * Np);
        PAMD_CU(c, cudaMemcpyAsync(fo.data(), c->b.fout, fo.size() * 4, cudaMemcpyDeviceToHost, c->stream));
    }
    if (E) PAMD_CU(c, cudaMemcpyAsync(E, cur_E(c), 8 * (size_t)R, cudaMemcpyDeviceToHost, c->stream));
    PAMD_CU(c, cudaStreamSynchronize(c->stream));
    for (long long k = 0; k < R && f; ++k)
        for (int i = 0; i < N; ++i)
            for (int q = 0; q < 3; ++q)
                f[((size_t)k * N + i) * 3 + q] = fo64.empty() ? (double)fo[(size_t)k * 3 * Np + (size_t)q * Np + i]
                                                               : fo64[(size_t)k * 3 * Np + (size_t)q * Np + i];
    return read_status(c);
}

int pamd_autotune(pamd_ctx* c, int32_t theta_probe, pamd_tune* out) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (is_batch(c)) return fail(PAMD_EINVAL, "batch context: call this on pamd_batch_sub(ctx, m)");
    if (theta_probe < 1 || theta_probe > 1000) return fail(PAMD_EINVAL, "theta_probe must be 1..1000");
    return autotune_with(c, theta_probe, TuneLimits{1, 8, true, true, {2, 4, 8}, 0}, out);
}

}  // extern "C"

namespace {

int autotune_with(pamd_ctx* c, int32_t theta_probe, const TuneLimits& lim, pamd_tune* out) {
    int rc = PAMD_OK;
    // the shapes tuned are those of the exact-force kernel
    struct ModelDetach {
        pamd_ctx* c;
        pamd_mlp* m;
        ~ModelDetach() { c->mlp = m; }
    } detach{c, c->mlp};
    c->mlp = nullptr;
    if (is_f64(c)) {  // one fixed shape (a warp per replica)
        if (out) *out = pamd_tune{32, (c->N + 31) / 32, 4, 1, 0, 0.0};
        return PAMD_OK;
    }
    const pamd_topology t = c->host_top.view();
    const int chain = (int)is_linear_chain(&t);
    const TuneKey key{c->N, c->R, chain, lim.key_tag ? lim.key_tag : c->lanes_req,
                      lim.packed_ok ? c->pair_arith : PAMD_PAIRS_SCALAR};
    TuneShape best_shape{0, 0, 0};
    double best_ms = 0.0;
    bool cached = tune_cache_lookup(key, &best_shape);
    std::vector<unsigned char> blob;
    TopoLayout lay;
    auto apply = [&](const TuneShape& sh) -> int {
        int r = build_topology(&t, sh.L, &lay, blob);
        if (r) return r;
        if (blob.size() > c->topo_cap) {
            void* p = dalloc(c, blob.size());
            if (!p) return fail(PAMD_ENOMEM, "topology table");
            c->b.topo = (unsigned char*)p;
            c->topo_cap = blob.size();
        }
        PAMD_CU(c, cudaMemcpyAsync(c->b.topo, blob.data(), blob.size(), cudaMemcpyHostToDevice, c->stream));
        PAMD_CU(c, cudaStreamSynchronize(c->stream));
        return set_launch_shape(c, lay, sh.W, sh.variant);
    };
    if (!cached) {
        // scratch copy of the population; per-replica outputs go to scratch too
        const size_t st_bytes = state_bytes(c);
        float* scratch = c->cur_is_alt ? c->b.state : c->b.state_alt;
        double* e_scr = c->cur_is_alt ? c->b.E : c->b.E_alt;
        double* ke_scr = reinterpret_cast<double*>(c->b.W);
        double* rg_scr = reinterpret_cast<double*>(c->b.C);
        cudaEvent_t e0, e1;
        PAMD_CU(c, cudaEventCreate(&e0));
        PAMD_CU(c, cudaEventCreate(&e1));
        double best = 1e300;
        std::vector<TuneShape> shapes;
        for (int b = lim.bmin; b <= lim.bmax; ++b) {
            int l = c->lanes_req ? c->lanes_req : (c->N + b - 1) / b;
            if (l > 32) continue;
            const int bb = (c->N + l - 1) / l;
            if (bb < lim.bmin || bb > lim.bmax) continue;
            l = (c->N + bb - 1) / bb;
            for (int var = kVarScalar; var <= kVarPacked; ++var) {
                if (var == kVarPaired && (!lim.paired_ok || bb < 2 || bb > 4)) continue;
                if (var == kVarPacked && (!lim.packed_ok || !chain || bb < 3 || bb > 8)) continue;
                if (var == kVarScalar && c->pair_arith == PAMD_PAIRS_PACKED) continue;
                if (var == kVarPacked && c->pair_arith == PAMD_PAIRS_SCALAR) continue;
                for (int w : lim.warps) {
                    bool dup = false;
                    for (auto& s2 : shapes) dup = dup || (s2.L == l && s2.W == w && s2.variant == var);
                    if (!dup) shapes.push_back({l, w, var});
                }
            }
        }
        int err = PAMD_OK;
        for (auto& sh : shapes) {
            if ((err = apply(sh))) {
                if (err == PAMD_EUNSUPPORTED) { err = PAMD_OK; continue; }
                break;
            }
            if (c->warps_per_block != sh.W) continue;  // shared memory capped it
            cudaMemcpyAsync(scratch, cur_state(c), st_bytes, cudaMemcpyDeviceToDevice, c->stream);
            if ((err = launch_prop_on(c, scratch, e_scr, ke_scr, rg_scr, 1, 0.001, 300.0, nullptr,
                                      c->step, nullptr)))
                break;
            cudaEventRecord(e0, c->stream);
            if ((err = launch_prop_on(c, scratch, e_scr, ke_scr, rg_scr, theta_probe, 0.001, 300.0,
                                      nullptr, c->step, nullptr)))
                break;
            cudaEventRecord(e1, c->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                err = cuda_fail(c, cudaGetLastError(), "autotune");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                best_shape = sh;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (err) return err;
        if (best == 1e300) return fail(PAMD_EUNSUPPORTED, "no feasible launch shape");
        best_ms = best;
        tune_cache_store(key, best_shape);
    }
    if ((rc = apply(best_shape))) return rc;
    if (c->graph_exec) {  // captured launches carry the old shape
        cudaGraphExecDestroy(c->graph_exec);
        c->graph_exec = nullptr;
        c->graph_key = GraphKey{};
    }
    if (out) {
        out->lanes_per_replica = c->lay.lanes;
        out->atoms_per_lane = c->lay.per_lane;
        out->warps_per_block = c->warps_per_block;
        out->replicas_per_lane = c->lay.paired ? 2 : 1;
        out->pair_arith = c->lay.packed ? PAMD_PAIRS_PACKED : PAMD_PAIRS_SCALAR;
        out->from_cache = cached ? 1 : 0;
        out->ms = best_ms;
    }
    return PAMD_OK;
}

}  // namespace

extern "C" {

int pamd_get_counters(pamd_ctx* c, uint32_t* step, uint32_t* ridx, double* sum_lnQ) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (is_batch(c)) return fail(PAMD_EINVAL, "batch context: call this on pamd_batch_sub(ctx, m)");
    if (step) *step = c->step;
    if (ridx) *ridx = c->resample_index;
    if (sum_lnQ) {
        PAMD_CU(c, cudaMemcpyAsync(sum_lnQ, &c->b.scal->sum_lnQ, 8, cudaMemcpyDeviceToHost, c->stream));
        PAMD_CU(c, cudaStreamSynchronize(c->stream));
    }
    return PAMD_OK;
}

int pamd_set_counters(pamd_ctx* c, uint32_t step, uint32_t ridx, double sum_lnQ) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (is_batch(c)) return fail(PAMD_EINVAL, "batch context: call this on pamd_batch_sub(ctx, m)");
    if (!std::isfinite(sum_lnQ)) return fail(PAMD_EINVAL, "sum_lnQ must be finite");
    c->step = step;
    c->resample_index = ridx;
    PAMD_CU(c, cudaMemcpyAsync(&c->b.scal->sum_lnQ, &sum_lnQ, 8, cudaMemcpyHostToDevice, c->stream));
    PAMD_CU(c, cudaStreamSynchronize(c->stream));
    return PAMD_OK;
}

int pamd_info(pamd_ctx* c, int64_t* R, int32_t* n_atoms, int32_t* lanes, int32_t* per_lane, int32_t* rpb) {
    if (!c) return fail(PAMD_EINVAL, "null context");
    if (is_batch(c)) {  // total replicas, largest molecule; shapes are per molecule
        if (R) *R = c->R;
        if (n_atoms) *n_atoms = c->N;
        if (lanes) *lanes = 0;
        if (per_lane) *per_lane = 0;
        if (rpb) *rpb = 0;
        return PAMD_OK;
    }
    if (R) *R = c->R;
    if (n_atoms) *n_atoms = c->N;
    if (lanes) *lanes = c->lay.lanes;
    if (per_lane) *per_lane = c->lay.per_lane;
    if (rpb) *rpb = c->rpb;
    return PAMD_OK;
}

int pamd_population_size(pamd_ctx* c, int64_t* live, int64_t* capacity) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (is_batch(c)) return fail(PAMD_EINVAL, "batch context: call this on pamd_batch_sub(ctx, m)");
    int64_t n = c->R;
    if (c->variable) {
        uint32_t v = 0;
        PAMD_CU(c, cudaMemcpyAsync(&v, c->b.counters + 2, sizeof(v), cudaMemcpyDeviceToHost, c->stream));
        PAMD_CU(c, cudaStreamSynchronize(c->stream));
        n = v;
    }
    if (live) *live = n;
    if (capacity) *capacity = c->R;
    return PAMD_OK;
}

int pamd_get_shape(pamd_ctx* c, pamd_tune* out) {
    if (!c || !out) return fail(PAMD_EINVAL, "null argument");
    if (is_batch(c)) return fail(PAMD_EINVAL, "batch context: call this on pamd_batch_sub(ctx, m)");
    *out = pamd_tune{};
    out->lanes_per_replica = c->lay.lanes;
    out->atoms_per_lane = c->lay.per_lane;
    out->warps_per_block = c->warps_per_block;
    out->replicas_per_lane = c->lay.paired ? 2 : 1;
    out->pair_arith = c->lay.packed ? PAMD_PAIRS_PACKED : PAMD_PAIRS_SCALAR;
    return PAMD_OK;
}

int64_t pamd_launch_count(pamd_ctx* c) {
    if (!c) return -1;
    long long n = c->launches;
    for (pamd_ctx* sub : c->subs) n += sub->launches;
    return n;
}

int pamd_sync(pamd_ctx* c) {
    int rc = check_ctx(c);
    if (rc) return rc;
    PAMD_CU(c, cudaStreamSynchronize(c->stream));
    return PAMD_OK;
}

}  // extern "C"

// ---- checkpoint files ------------------------------------------------------
//
// Layout (native byte order): 8-byte magic, then a header of fixed-size
// fields, then the payload, then an FNV-1a 64 checksum of header and payload.

namespace {

constexpr char kCkptMagic[8] = {'P', 'A', 'M', 'D', 'C', 'K', 'P', '1'};

struct CkptHeader {
    uint32_t version;
    int32_t precision;
    int64_t R;
    int32_t N, Np;
    uint64_t seed;
    uint32_t step, resample_index;
    double sum_lnQ;
    int32_t mol, pad_;
    uint64_t topology_hash;
};

uint64_t fnv1a(const void* data, size_t n, uint64_t h = 1469598103934665603ull) {
    const unsigned char* b = static_cast<const unsigned char*>(data);
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

uint64_t topology_hash(const HostTopology& t) {
    uint64_t h = fnv1a(&t.n_atoms, sizeof(t.n_atoms));
    auto mix = [&](const auto& v) {
        if (!v.empty()) h = fnv1a(v.data(), v.size() * sizeof(v[0]), h);
        const uint64_t n = v.size();
        h = fnv1a(&n, sizeof(n), h);
    };
    mix(t.mass); mix(t.charge); mix(t.sigma); mix(t.epsilon);
    mix(t.bond); mix(t.bond_r0); mix(t.bond_k); mix(t.angle); mix(t.angle_t0); mix(t.angle_k);
    mix(t.dihedral); mix(t.dih_n); mix(t.dih_k); mix(t.dih_phase); mix(t.excl); mix(t.pair14);
    h = fnv1a(&t.scale14_lj, sizeof(double), h);
    h = fnv1a(&t.scale14_coul, sizeof(double), h);
    return h;
}

}  // namespace

extern "C" {

int pamd_checkpoint(pamd_ctx* c, const char* path) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (c->variable) return fail(PAMD_EUNSUPPORTED, "not available with a variable population size");
    if (is_batch(c)) return fail(PAMD_EUNSUPPORTED, "checkpoint a batch molecule by molecule (pamd_batch_sub)");
    if (!path) return fail(PAMD_EINVAL, "null path");
    CkptHeader h{};
    h.version = 1;
    h.precision = c->precision;
    h.R = c->R;
    h.N = c->N;
    h.Np = c->Np;
    h.seed = c->seed;
    h.step = c->step;
    h.resample_index = c->resample_index;
    h.mol = c->mol;
    h.topology_hash = topology_hash(c->host_top);
    std::vector<unsigned char> st(state_bytes(c));
    std::vector<double> E((size_t)c->R);
    std::vector<int32_t> fam((size_t)c->R);
    PAMD_CU(c, cudaMemcpyAsync(&h.sum_lnQ, &c->b.scal->sum_lnQ, 8, cudaMemcpyDeviceToHost, c->stream));
    PAMD_CU(c, cudaMemcpyAsync(st.data(), cur_state(c), st.size(), cudaMemcpyDeviceToHost, c->stream));
    PAMD_CU(c, cudaMemcpyAsync(E.data(), cur_E(c), 8 * E.size(), cudaMemcpyDeviceToHost, c->stream));
    PAMD_CU(c, cudaMemcpyAsync(fam.data(), cur_fam(c), 4 * fam.size(), cudaMemcpyDeviceToHost, c->stream));
    PAMD_CU(c, cudaStreamSynchronize(c->stream));
    uint64_t sum = fnv1a(&h, sizeof(h));
    sum = fnv1a(st.data(), st.size(), sum);
    sum = fnv1a(E.data(), 8 * E.size(), sum);
    sum = fnv1a(fam.data(), 4 * fam.size(), sum);
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "wb");
    if (!f) return fail(PAMD_EINVAL, std::string("cannot write ") + tmp);
    bool ok = std::fwrite(kCkptMagic, 1, 8, f) == 8 && std::fwrite(&h, sizeof(h), 1, f) == 1 &&
              std::fwrite(st.data(), 1, st.size(), f) == st.size() &&
              std::fwrite(E.data(), 8, E.size(), f) == E.size() &&
              std::fwrite(fam.data(), 4, fam.size(), f) == fam.size() &&
              std::fwrite(&sum, sizeof(sum), 1, f) == 1;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return fail(PAMD_EINVAL, std::string("cannot write ") + path);
    }
    return PAMD_OK;
}

int pamd_restore(pamd_ctx* c, const char* path) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (c->variable) return fail(PAMD_EUNSUPPORTED, "not available with a variable population size");
    if (is_batch(c)) return fail(PAMD_EUNSUPPORTED, "restore a batch molecule by molecule (pamd_batch_sub)");
    if (!path) return fail(PAMD_EINVAL, "null path");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(PAMD_EINVAL, std::string("cannot read ") + path);
    char magic[8];
    CkptHeader h{};
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kCkptMagic, 8) == 0 &&
              std::fread(&h, sizeof(h), 1, f) == 1;
    if (!ok || h.version != 1) {
        std::fclose(f);
        return fail(PAMD_EINVAL, std::string(path) + ": not a checkpoint of this library");
    }
    if (h.precision != c->precision || h.R != c->R || h.N != c->N || h.Np != c->Np ||
        h.topology_hash != topology_hash(c->host_top)) {
        std::fclose(f);
        return fail(PAMD_EINVAL, std::string(path) + ": checkpoint of another population "
                                 "(precision, R, atoms or topology differ)");
    }
    std::vector<unsigned char> st(state_bytes(c));
    std::vector<double> E((size_t)c->R);
    std::vector<int32_t> fam((size_t)c->R);
    uint64_t sum_file = 0;
    ok = std::fread(st.data(), 1, st.size(), f) == st.size() &&
         std::fread(E.data(), 8, E.size(), f) == E.size() &&
         std::fread(fam.data(), 4, fam.size(), f) == fam.size() &&
         std::fread(&sum_file, sizeof(sum_file), 1, f) == 1;
    std::fclose(f);
    uint64_t sum = fnv1a(&h, sizeof(h));
    sum = fnv1a(st.data(), st.size(), sum);
    sum = fnv1a(E.data(), 8 * E.size(), sum);
    sum = fnv1a(fam.data(), 4 * fam.size(), sum);
    if (!ok || sum != sum_file) return fail(PAMD_EINVAL, std::string(path) + ": truncated or corrupt checkpoint");
    for (int32_t v : fam)
        if (v < 0 || v >= c->R) return fail(PAMD_EINVAL, std::string(path) + ": family ids out of range");
    // the restored population goes to the main buffers
    c->cur_is_alt = false;
    PAMD_CU(c, cudaMemcpyAsync(c->b.state, st.data(), st.size(), cudaMemcpyHostToDevice, c->stream));
    PAMD_CU(c, cudaMemcpyAsync(c->b.E, E.data(), 8 * E.size(), cudaMemcpyHostToDevice, c->stream));
    PAMD_CU(c, cudaMemcpyAsync(c->b.fam, fam.data(), 4 * fam.size(), cudaMemcpyHostToDevice, c->stream));
    PAMD_CU(c, cudaMemcpyAsync(&c->b.scal->sum_lnQ, &h.sum_lnQ, 8, cudaMemcpyHostToDevice, c->stream));
    PAMD_CU(c, cudaStreamSynchronize(c->stream));
    c->seed = h.seed;
    c->step = h.step;
    c->resample_index = h.resample_index;
    return PAMD_OK;
}

int pamd_set_force_model(pamd_ctx* c, pamd_mlp* m) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (c->variable) return fail(PAMD_EUNSUPPORTED, "not available with a variable population size");
    if (is_batch(c) || is_f64(c))
        return fail(PAMD_EUNSUPPORTED, "force models need a single-molecule mixed-precision context");
    if (m) {
        if (m->N != c->N) return fail(PAMD_EINVAL, "force model is for another atom count");
        if (m->broken) return fail(PAMD_ESTATE, "force model unusable after an earlier CUDA error");
        PAMD_CU(c, cudaStreamSynchronize(c->stream));
        if ((rc = mlp_ensure_work(m, c->R, false))) return rc;
        PAMD_CU(c, cudaStreamSynchronize(m->stream));
    }
    c->mlp = m;
    return PAMD_OK;
}

void pamd_destroy(pamd_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (pamd_ctx* sub : c->subs) pamd_destroy(sub);
    c->subs.clear();
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    for (cudaStream_t s : c->group_streams) cudaStreamDestroy(s);
    for (cudaEvent_t e : c->group_events) cudaEventDestroy(e);
    if (c->fork_event) cudaEventDestroy(c->fork_event);
    free_all(c);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

}  // extern "C"
