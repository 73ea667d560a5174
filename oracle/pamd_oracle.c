/*
 * pamd_oracle.c -- plain FP64 CPU oracle for population-annealing molecular
 * dynamics (PAMD), Christiansen, Weigel & Janke, arXiv:1806.06016.
 *
 * TEST INFRASTRUCTURE.  This library exists to check the CUDA library and to
 * serve as the timed CPU baseline.  Only the test suite, the smoke check and
 * the benchmark's CPU-baseline / reference legs load it.  It shares no code,
 * header, table or constant generator with the CUDA library; the only common
 * ground is the seeded input generator (topologies, schedules) that both
 * receive as plain arrays.
 *
 * It follows the paper's statement of the method in order (PAMD scheme,
 * steps 1-5): set up R copies at T0, resample with relative Boltzmann weights,
 * run theta MD steps per copy, measure population averages, repeat.
 * Everything is FP64, summations run in a fixed sequential order, and the only
 * parallelism is a split of the replicas over POSIX threads during the MD
 * steps (replicas are independent there; see the paragraph on parallelisation
 * over independent replicas in the introduction).
 *
 * Readings of points the paper leaves open:
 *   - MD engine: BAOAB Langevin splitting (Leimkuhler & Matthews 2013) with
 *     friction gamma; the paper's own integrator is a velocity-Verlet-type
 *     scheme with a Langevin thermostat and a per-replica seed.
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11) keyed on the run
 *     seed, counter = (atom, replica slot, step, purpose | molecule << 8).
 *     Normals: Box-Muller on 23-bit uniforms u = (top23 + 0.5) * 2^-23, which
 *     binary32 and binary64 both represent exactly.
 *   - Multinomial resampling is realised with integer weights
 *     W_j = floor(2^s * exp(a_j - max a)), s = 63 - ceil(log2 R), an inclusive
 *     prefix sum C and R targets t_k = floor(u_k * C_total / 2^64) from 64-bit
 *     Philox uniforms; ancestor = first j with C_j > t_k.  The exponential in
 *     W uses exp_det, a Cody-Waite reduction plus a degree-13 Taylor
 *     polynomial evaluated with explicit fused multiply-adds, so that it gives
 *     the same bits on every IEEE machine.
 *   - After resampling positions are recentred on the centre of mass and
 *     velocities scaled by sqrt(T_i / T_{i-1}) (PAMD scheme, step 2).
 *   - Standard errors: jackknife over 64 bins, bin = family id mod 64 (family
 *     id = replica slot at T0), following the paper's paragraph on error
 *     estimates by binning.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "pamd_oracle.h"

#define ORC_KB 0.008314462618   /* Boltzmann constant, kJ/mol/K */
#define ORC_KE 138.935458       /* Coulomb constant, kJ mol^-1 nm e^-2 */

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11, Sec. 4 "Philox").       */
/* Ten rounds of the 4x32 Philox S-P network; the key is bumped by the Weyl   */
/* constants between rounds.                                                  */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox_keyed(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                         uint32_t out[4]) {
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* Uniform in (0,1) from the top 23 bits of a 32-bit draw (exact in binary32). */
static double u23(uint32_t u) { return ((double)(u >> 9) + 0.5) * 0x1p-23; }

/* Three standard normals for (atom, slot, step, purpose) by Box-Muller. */
void orc_normal3(uint64_t seed, uint32_t atom, uint32_t slot, uint32_t step, uint32_t purpose,
                 double z[3]) {
    uint32_t o[4];
    philox_keyed(seed, atom, slot, step, purpose, o);
    const double two_pi = 6.283185307179586476925286766559;
    double r0 = sqrt(-2.0 * log(u23(o[0])));
    double r1 = sqrt(-2.0 * log(u23(o[2])));
    z[0] = r0 * cos(two_pi * u23(o[1]));
    z[1] = r0 * sin(two_pi * u23(o[1]));
    z[2] = r1 * cos(two_pi * u23(o[3]));
}

/* ------------------------------------------------------------------------- */
/* exp_det: e^x for x <= 709 by Cody & Waite (1980) argument reduction        */
/* x = k ln2 + r, |r| <= ln2/2, and the Taylor series of e^r to degree 13      */
/* (truncation error < 2^-57 relative) in Horner form with explicit fma.      */
/* ------------------------------------------------------------------------- */
static double g_inv_fact[14];
static pthread_once_t g_fact_once = PTHREAD_ONCE_INIT;
static void init_inv_fact(void) {
    double f = 1.0;
    for (int n = 0; n < 14; ++n) {
        if (n > 0) f *= (double)n; /* n! is exact in binary64 for n <= 18 */
        g_inv_fact[n] = 1.0 / f;
    }
}

double orc_exp_det(double x) {
    pthread_once(&g_fact_once, init_inv_fact);
    if (x < -708.0) return 0.0;
    if (x > 709.0) return INFINITY;
    const double inv_ln2 = 0x1.71547652b82fep+0;
    const double ln2_hi = 0x1.62e42fee00000p-1;  /* ln2 to 32 significant bits */
    const double ln2_lo = 0x1.a39ef35793c76p-33; /* ln2 - ln2_hi */
    double kf = nearbyint(x * inv_ln2);
    double r = fma(-kf, ln2_hi, x);
    r = fma(-kf, ln2_lo, r);
    double p = g_inv_fact[13];
    for (int n = 12; n >= 0; --n) p = fma(p, r, g_inv_fact[n]);
    int k = (int)kf;
    union { uint64_t u; double d; } two_k;
    two_k.u = (uint64_t)(k + 1023) << 52;
    return p * two_k.d;
}

/* ------------------------------------------------------------------------- */
/* Force field                                                               */
/* ------------------------------------------------------------------------- */

/* Nonbonded pair kinds, from the exclusion and 1-4 lists. */
enum { PAIR_FULL = 0, PAIR_EXCL = 1, PAIR_14 = 2 };

static unsigned char* pair_kind_matrix(const orc_topology* t) {
    int n = t->n_atoms;
    unsigned char* m = (unsigned char*)calloc((size_t)n * n, 1);
    if (!m) return NULL;
    for (int p = 0; p < t->n_pair14; ++p) {
        int i = t->pair14[2 * p], j = t->pair14[2 * p + 1];
        m[i * n + j] = m[j * n + i] = PAIR_14;
    }
    for (int p = 0; p < t->n_excl; ++p) { /* an exclusion wins over a 1-4 entry */
        int i = t->excl[2 * p], j = t->excl[2 * p + 1];
        m[i * n + j] = m[j * n + i] = PAIR_EXCL;
    }
    return m;
}

static inline void sub3(const double* a, const double* b, double* d) {
    d[0] = a[0] - b[0]; d[1] = a[1] - b[1]; d[2] = a[2] - b[2];
}
static inline double dot3(const double* a, const double* b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static inline void cross3(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Torsion angle of (i, j, k, l), IUPAC sign convention, in (-pi, pi]. */
double orc_dihedral_angle(const double* xi, const double* xj, const double* xk, const double* xl) {
    double b1[3], b2[3], b3[3], n1[3], n2[3], m[3];
    sub3(xj, xi, b1);
    sub3(xk, xj, b2);
    sub3(xl, xk, b3);
    cross3(b1, b2, n1);
    cross3(b2, b3, n2);
    double lb2 = sqrt(dot3(b2, b2));
    double y = lb2 * dot3(b1, n2);
    double x = dot3(n1, n2);
    (void)m;
    return atan2(y, x);
}

/*
 * Potential energy (kJ/mol) and forces (kJ/mol/nm) of one configuration.
 *   bonds:      1/2 k (r - r0)^2
 *   angles:     1/2 k (theta - theta0)^2
 *   dihedrals:  k (1 + cos(n phi - phase))
 *   nonbonded:  for every pair i<j not excluded, with s = scale14 for 1-4
 *               pairs and 1 otherwise:
 *               s_lj * 4 eps [(sig/r)^12 - (sig/r)^6] + s_c * k_e q_i q_j / r,
 *               sig = (sig_i + sig_j)/2, eps = sqrt(eps_i eps_j).
 * x, f: [N][3].  f may be NULL.  terms (may be NULL) receives
 * {bond, angle, dihedral, lj, coulomb}.
 */
double orc_energy_forces(const orc_topology* t, const double* x, double* f, double* terms) {
    int n = t->n_atoms;
    double e_bond = 0, e_angle = 0, e_dih = 0, e_lj = 0, e_c = 0;
    if (f) memset(f, 0, sizeof(double) * 3 * (size_t)n);

    for (int b = 0; b < t->n_bonds; ++b) {
        int i = t->bond[2 * b], j = t->bond[2 * b + 1];
        double d[3];
        sub3(&x[3 * i], &x[3 * j], d);
        double r = sqrt(dot3(d, d));
        double r0 = t->bond_r0[b], k = t->bond_k[b];
        e_bond += 0.5 * k * (r - r0) * (r - r0);
        if (f) {
            /* dE/dx_i = k (r - r0) d / r */
            double g = (r0 == 0.0) ? k : k * (r - r0) / r;
            for (int c = 0; c < 3; ++c) {
                f[3 * i + c] -= g * d[c];
                f[3 * j + c] += g * d[c];
            }
        }
    }

    for (int a = 0; a < t->n_angles; ++a) {
        int i = t->angle[3 * a], j = t->angle[3 * a + 1], k = t->angle[3 * a + 2];
        double u[3], w[3], uxw[3];
        sub3(&x[3 * i], &x[3 * j], u);
        sub3(&x[3 * k], &x[3 * j], w);
        cross3(u, w, uxw);
        double s = sqrt(dot3(uxw, uxw)), c = dot3(u, w);
        double theta = atan2(s, c);
        double dth = theta - t->angle_t0[a];
        e_angle += 0.5 * t->angle_k[a] * dth * dth;
        if (f) {
            /* dtheta/du = -(w - (u.w) u / |u|^2) / |u x w|, likewise for w */
            double g = t->angle_k[a] * dth; /* dE/dtheta */
            double uu = dot3(u, u), ww = dot3(w, w);
            for (int q = 0; q < 3; ++q) {
                double dthu = -(w[q] - c * u[q] / uu) / s;
                double dthw = -(u[q] - c * w[q] / ww) / s;
                f[3 * i + q] -= g * dthu;
                f[3 * k + q] -= g * dthw;
                f[3 * j + q] += g * (dthu + dthw);
            }
        }
    }

    for (int d = 0; d < t->n_dihedrals; ++d) {
        int i = t->dihedral[4 * d], j = t->dihedral[4 * d + 1];
        int k = t->dihedral[4 * d + 2], l = t->dihedral[4 * d + 3];
        double phi = orc_dihedral_angle(&x[3 * i], &x[3 * j], &x[3 * k], &x[3 * l]);
        double kd = t->dih_k[d], nn = (double)t->dih_n[d], ph = t->dih_phase[d];
        e_dih += kd * (1.0 + cos(nn * phi - ph));
        if (f) {
            /* Gradient of phi after Blondel & Karplus (1996): with
             * F = x_i - x_j, G = x_j - x_k, H = x_l - x_k, A = F x G, B = H x G,
             * dphi/dx_i = -|G|/|A|^2 A, dphi/dx_l = |G|/|B|^2 B, and the inner
             * atoms take the rest so that the total is translation invariant. */
            double F[3], G[3], H[3], A[3], B[3];
            sub3(&x[3 * i], &x[3 * j], F);
            sub3(&x[3 * j], &x[3 * k], G);
            sub3(&x[3 * l], &x[3 * k], H);
            cross3(F, G, A);
            cross3(H, G, B);
            double AA = dot3(A, A), BB = dot3(B, B), lg = sqrt(dot3(G, G));
            double fg = dot3(F, G), hg = dot3(H, G);
            double dEdphi = -kd * nn * sin(nn * phi - ph);
            for (int q = 0; q < 3; ++q) {
                double gi = -lg / AA * A[q];
                double gl = lg / BB * B[q];
                double gj = lg / AA * A[q] + fg / (AA * lg) * A[q] - hg / (BB * lg) * B[q];
                double gk = -fg / (AA * lg) * A[q] + hg / (BB * lg) * B[q] - lg / BB * B[q];
                f[3 * i + q] -= dEdphi * gi;
                f[3 * j + q] -= dEdphi * gj;
                f[3 * k + q] -= dEdphi * gk;
                f[3 * l + q] -= dEdphi * gl;
            }
        }
    }

    unsigned char* kind = pair_kind_matrix(t);
    if (!kind && n > 0) return NAN;
    for (int i = 0; i < n; ++i) {
        for (int j = i + 1; j < n; ++j) {
            int kd = kind[i * n + j];
            if (kd == PAIR_EXCL) continue;
            double s_lj = (kd == PAIR_14) ? t->scale14_lj : 1.0;
            double s_c = (kd == PAIR_14) ? t->scale14_coul : 1.0;
            double d[3];
            sub3(&x[3 * i], &x[3 * j], d);
            double r2 = dot3(d, d), r = sqrt(r2);
            double sig = 0.5 * (t->sigma[i] + t->sigma[j]);
            double eps = sqrt(t->epsilon[i] * t->epsilon[j]);
            double sr6 = pow(sig / r, 6.0);
            double sr12 = sr6 * sr6;
            double qq = ORC_KE * t->charge[i] * t->charge[j];
            e_lj += s_lj * 4.0 * eps * (sr12 - sr6);
            e_c += s_c * qq / r;
            if (f) {
                /* -dE/dr divided by r, so that F_i = g * (x_i - x_j) */
                double g = s_lj * 24.0 * eps * (2.0 * sr12 - sr6) / r2 + s_c * qq / (r2 * r);
                for (int c = 0; c < 3; ++c) {
                    f[3 * i + c] += g * d[c];
                    f[3 * j + c] -= g * d[c];
                }
            }
        }
    }
    free(kind);
    if (terms) {
        terms[0] = e_bond; terms[1] = e_angle; terms[2] = e_dih; terms[3] = e_lj; terms[4] = e_c;
    }
    return e_bond + e_angle + e_dih + e_lj + e_c;
}

/* ------------------------------------------------------------------------- */
/* Population helpers                                                        */
/* ------------------------------------------------------------------------- */

static void recentre(const orc_topology* t, double* x) {
    int n = t->n_atoms;
    double c[3] = {0, 0, 0}, mt = 0;
    for (int i = 0; i < n; ++i) {
        for (int q = 0; q < 3; ++q) c[q] += t->mass[i] * x[3 * i + q];
        mt += t->mass[i];
    }
    for (int q = 0; q < 3; ++q) c[q] /= mt;
    for (int i = 0; i < n; ++i)
        for (int q = 0; q < 3; ++q) x[3 * i + q] -= c[q];
}

/* Step 1 of the PAMD scheme: R copies of the start geometry at T0 (recentred),
 * velocities drawn from the Maxwell-Boltzmann distribution at T0,
 * family id = slot. */
void orc_init(const orc_topology* t, int64_t R, double T0, uint64_t seed, int32_t mol,
              double* x, double* v, int32_t* fam) {
    int n = t->n_atoms;
    double* x0 = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    memcpy(x0, t->x0, sizeof(double) * 3 * (size_t)n);
    recentre(t, x0);
    for (int64_t k = 0; k < R; ++k) {
        memcpy(&x[(size_t)k * 3 * n], x0, sizeof(double) * 3 * (size_t)n);
        for (int i = 0; i < n; ++i) {
            double z[3];
            orc_normal3(seed, (uint32_t)i, (uint32_t)k, 0u, ORC_PURPOSE_INIT | ((uint32_t)mol << 8), z);
            double sd = sqrt(ORC_KB * T0 / t->mass[i]);
            for (int q = 0; q < 3; ++q) v[(size_t)k * 3 * n + 3 * i + q] = sd * z[q];
        }
        fam[k] = (int32_t)k;
    }
    free(x0);
}

/* Step 3 of the PAMD scheme for one replica: theta BAOAB Langevin steps
 * (Leimkuhler & Matthews 2013) at temperature T, friction gamma.
 *   B: v += dt/2 F/m;  A: x += dt/2 v;  O: v = c1 v + sqrt((1-c1^2) kT/m) xi;
 *   A: x += dt/2 v;    F = F(x);        B: v += dt/2 F/m;     c1 = exp(-gamma dt).
 * xi from Philox(seed; atom, slot, step0 + s, NOISE | mol << 8).
 * Returns the potential energy after the last step. */
static double propagate_one(const orc_topology* t, double* x, double* v, double* f, int64_t slot,
                            int32_t theta, double dt, double T, double gamma, uint64_t seed,
                            uint32_t step0, int32_t mol) {
    int n = t->n_atoms;
    double c1 = exp(-gamma * dt);
    double c2 = sqrt(1.0 - c1 * c1);
    double kT = ORC_KB * T;
    orc_energy_forces(t, x, f, NULL);
    for (int32_t s = 0; s < theta; ++s) {
        for (int i = 0; i < n; ++i) {
            double im = 1.0 / t->mass[i];
            double sd = c2 * sqrt(kT * im);
            double z[3];
            orc_normal3(seed, (uint32_t)i, (uint32_t)slot, step0 + (uint32_t)s,
                        ORC_PURPOSE_NOISE | ((uint32_t)mol << 8), z);
            for (int q = 0; q < 3; ++q) {
                double* vq = &v[3 * i + q];
                double* xq = &x[3 * i + q];
                *vq += 0.5 * dt * f[3 * i + q] * im; /* B */
                *xq += 0.5 * dt * (*vq);             /* A */
                *vq = c1 * (*vq) + sd * z[q];        /* O */
                *xq += 0.5 * dt * (*vq);             /* A */
            }
        }
        orc_energy_forces(t, x, f, NULL);
        for (int i = 0; i < n; ++i) {
            double im = 1.0 / t->mass[i];
            for (int q = 0; q < 3; ++q) v[3 * i + q] += 0.5 * dt * f[3 * i + q] * im; /* B */
        }
    }
    return orc_energy_forces(t, x, NULL, NULL);
}

typedef struct {
    const orc_topology* t;
    double *x, *v, *E;
    const int64_t* slots; /* noise slot of each replica, or NULL for its index */
    int64_t lo, hi;
    int32_t theta, mol;
    double dt, T, gamma;
    uint64_t seed;
    uint32_t step0;
} prop_job;

static void* prop_worker(void* arg) {
    prop_job* j = (prop_job*)arg;
    int n = j->t->n_atoms;
    double* f = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    for (int64_t k = j->lo; k < j->hi; ++k) {
        int64_t slot = j->slots ? j->slots[k] : k;
        double e = propagate_one(j->t, &j->x[(size_t)k * 3 * n], &j->v[(size_t)k * 3 * n], f, slot,
                                 j->theta, j->dt, j->T, j->gamma, j->seed, j->step0, j->mol);
        if (j->E) j->E[k] = e;
    }
    free(f);
    return NULL;
}

/* theta MD steps for R replicas; replica k uses noise slot slots[k] (or k when
 * slots is NULL).  x, v: [R][N][3]; E (may be NULL): [R]. */
void orc_propagate_slots(const orc_topology* t, int64_t R, const int64_t* slots, double* x,
                         double* v, double* E, int32_t theta, double dt, double T, double gamma,
                         uint64_t seed, uint32_t step0, int32_t mol, int32_t n_threads) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > R) n_threads = (int32_t)(R > 0 ? R : 1);
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * n_threads);
    prop_job* jobs = (prop_job*)malloc(sizeof(prop_job) * n_threads);
    for (int w = 0; w < n_threads; ++w) {
        prop_job jb = {t, x, v, E, slots, R * w / n_threads, R * (w + 1) / n_threads, theta, mol,
                       dt, T, gamma, seed, step0};
        jobs[w] = jb;
        if (n_threads == 1) prop_worker(&jobs[w]);
        else pthread_create(&th[w], NULL, prop_worker, &jobs[w]);
    }
    if (n_threads > 1)
        for (int w = 0; w < n_threads; ++w) pthread_join(th[w], NULL);
    free(th);
    free(jobs);
}

/* theta MD steps for every replica (slot = index). */
void orc_propagate(const orc_topology* t, int64_t R, double* x, double* v, double* E,
                   int32_t theta, double dt, double T, double gamma, uint64_t seed,
                   uint32_t step0, int32_t mol, int32_t n_threads) {
    orc_propagate_slots(t, R, NULL, x, v, E, theta, dt, T, gamma, seed, step0, mol, n_threads);
}

/* Potential energy of every replica (FP64). */
void orc_energies(const orc_topology* t, int64_t R, const double* x, double* E) {
    int n = t->n_atoms;
    for (int64_t k = 0; k < R; ++k) E[k] = orc_energy_forces(t, &x[(size_t)k * 3 * n], NULL, NULL);
}

/* ------------------------------------------------------------------------- */
/* Resampling (PAMD scheme, step 2, and the paragraph on multinomial draws)   */
/* ------------------------------------------------------------------------- */

int32_t orc_weight_shift(int64_t R) {
    int32_t bits = 0;
    while (((int64_t)1 << bits) < R) ++bits;
    return 63 - bits;
}

/* ln Q with Q = (1/R) sum_j exp(-(beta_next - beta_prev) E_j), and the integer
 * weights W_j = floor(2^s exp_det(a_j - max a)), a_j = -(beta_next - beta_prev) E_j.
 * Returns ln Q; W may be NULL. */
double orc_resample_weights(const double* E, int64_t R, double T_prev, double T_next, uint64_t* W) {
    double dbeta = 1.0 / (ORC_KB * T_next) - 1.0 / (ORC_KB * T_prev);
    double m = -INFINITY;
    for (int64_t j = 0; j < R; ++j) {
        double a = -dbeta * E[j];
        if (a > m) m = a;
    }
    double S = 0.0;
    for (int64_t j = 0; j < R; ++j) S += exp(-dbeta * E[j] - m);
    if (W) {
        int32_t s = orc_weight_shift(R);
        double scale = ldexp(1.0, s);
        for (int64_t j = 0; j < R; ++j) W[j] = (uint64_t)floor(scale * orc_exp_det(-dbeta * E[j] - m));
    }
    return m + (log(S) - log((double)R));
}

/* First index j with C[j] > t (C inclusive prefix sums, non-decreasing). */
int64_t orc_ancestor(const uint64_t* C, int64_t R, uint64_t t) {
    int64_t lo = 0, hi = R; /* answer in [lo, hi) */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (C[mid] > t) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

/* 64-bit uniform for draw k of resampling step temp_index. */
uint64_t orc_resample_uniform(uint64_t seed, uint32_t k, uint32_t temp_index, int32_t mol) {
    uint32_t o[4];
    philox_keyed(seed, k, temp_index, 0u, ORC_PURPOSE_RESAMPLE | ((uint32_t)mol << 8), o);
    return (uint64_t)o[0] | ((uint64_t)o[1] << 32);
}

/* R multinomial draws with probabilities W_j / sum W: counts[j] = copies of j. */
void orc_multinomial_counts(const uint64_t* W, int64_t R, uint64_t seed, uint32_t temp_index,
                            int32_t mol, int32_t* counts) {
    uint64_t* C = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(R > 0 ? R : 1));
    uint64_t acc = 0;
    for (int64_t j = 0; j < R; ++j) {
        acc += W[j];
        C[j] = acc;
        counts[j] = 0;
    }
    for (int64_t k = 0; k < R; ++k) {
        uint64_t u = orc_resample_uniform(seed, (uint32_t)k, temp_index, mol);
        uint64_t t = (uint64_t)(((unsigned __int128)u * (unsigned __int128)acc) >> 64);
        counts[orc_ancestor(C, R, t)] += 1;
    }
    free(C);
}

/* New population: copies of ancestor j fill slots off_j .. off_j + n_j - 1
 * (ascending ancestor order).  Positions recentred, velocities scaled by
 * vscale = sqrt(T_next / T_prev), family ids and energies carried along. */
void orc_gather(const orc_topology* t, int64_t R, const int32_t* counts, const double* x,
                const double* v, const int32_t* fam, const double* E, double vscale,
                double* x_new, double* v_new, int32_t* fam_new, double* E_new) {
    int n = t->n_atoms;
    size_t rs = 3 * (size_t)n;
    int64_t k = 0;
    for (int64_t j = 0; j < R; ++j) {
        for (int32_t c = 0; c < counts[j]; ++c, ++k) {
            memcpy(&x_new[k * rs], &x[j * rs], sizeof(double) * rs);
            recentre(t, &x_new[k * rs]);
            for (size_t q = 0; q < rs; ++q) v_new[k * rs + q] = vscale * v[j * rs + q];
            fam_new[k] = fam[j];
            if (E_new) E_new[k] = E[j];
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Observables (PAMD scheme, step 4) with family-binned jackknife errors      */
/* ------------------------------------------------------------------------- */

double orc_kinetic(const orc_topology* t, const double* v) {
    double ek = 0;
    for (int i = 0; i < t->n_atoms; ++i) ek += 0.5 * t->mass[i] * dot3(&v[3 * i], &v[3 * i]);
    return ek;
}

/* Radius of gyration sqrt((1/N) sum |x_i - mean x|^2), unweighted. */
double orc_rgyr(const orc_topology* t, const double* x) {
    int n = t->n_atoms;
    double c[3] = {0, 0, 0};
    for (int i = 0; i < n; ++i)
        for (int q = 0; q < 3; ++q) c[q] += x[3 * i + q];
    for (int q = 0; q < 3; ++q) c[q] /= n;
    double s = 0;
    for (int i = 0; i < n; ++i) {
        double d[3];
        sub3(&x[3 * i], c, d);
        s += dot3(d, d);
    }
    return sqrt(s / n);
}

/* Jackknife standard error of the population mean over ORC_NBINS bins
 * (bin = family mod ORC_NBINS); empty bins are skipped. */
static double binned_se(const double* val, const int32_t* fam, int64_t R, double* mean_out) {
    double sum[ORC_NBINS] = {0};
    int64_t cnt[ORC_NBINS] = {0};
    double tot = 0;
    for (int64_t k = 0; k < R; ++k) {
        int b = (int)(fam[k] % ORC_NBINS);
        sum[b] += val[k];
        cnt[b] += 1;
        tot += val[k];
    }
    double mean = tot / (double)R;
    if (mean_out) *mean_out = mean;
    int nb = 0;
    double jk[ORC_NBINS];
    for (int b = 0; b < ORC_NBINS; ++b) {
        if (cnt[b] == 0 || cnt[b] == R) continue;
        jk[nb++] = (tot - sum[b]) / (double)(R - cnt[b]);
    }
    if (nb < 2) return 0.0;
    double jm = 0;
    for (int b = 0; b < nb; ++b) jm += jk[b];
    jm /= nb;
    double ss = 0;
    for (int b = 0; b < nb; ++b) ss += (jk[b] - jm) * (jk[b] - jm);
    return sqrt((double)(nb - 1) / nb * ss);
}

void orc_observables(const orc_topology* t, int64_t R, const double* x, const double* v,
                     const int32_t* fam, const double* E, orc_obs* o) {
    int n = t->n_atoms;
    double* ek = (double*)malloc(sizeof(double) * (size_t)R);
    double* rg = (double*)malloc(sizeof(double) * (size_t)R);
    double* rg2 = (double*)malloc(sizeof(double) * (size_t)R);
    for (int64_t k = 0; k < R; ++k) {
        ek[k] = orc_kinetic(t, &v[(size_t)k * 3 * n]);
        rg[k] = orc_rgyr(t, &x[(size_t)k * 3 * n]);
        rg2[k] = rg[k] * rg[k];
    }
    o->e_pot_se = binned_se(E, fam, R, &o->e_pot);
    o->e_kin_se = binned_se(ek, fam, R, &o->e_kin);
    o->rg_se = binned_se(rg, fam, R, &o->rg);
    o->rg2_se = binned_se(rg2, fam, R, &o->rg2);
    o->t_meas = 2.0 * o->e_kin / (3.0 * n * ORC_KB);
    /* number of distinct families */
    unsigned char* seen = (unsigned char*)calloc((size_t)R, 1);
    int64_t nf = 0;
    for (int64_t k = 0; k < R; ++k) {
        if (fam[k] >= 0 && fam[k] < R && !seen[fam[k]]) {
            seen[fam[k]] = 1;
            ++nf;
        }
    }
    o->n_families = nf;
    free(seen);
    free(ek);
    free(rg);
    free(rg2);
}

/* ------------------------------------------------------------------------- */
/* Whole anneal (PAMD scheme, steps 1-5)                                      */
/* ------------------------------------------------------------------------- */

/* T[0..K] (K resampling steps).  out[0..K].  x, v ([R][N][3]) receive the final
 * population; fam, E likewise ([R]).  resample = 0 turns resampling off
 * (copy counts all 1, the "anneal" control), velocities are still rescaled. */
int orc_anneal(const orc_topology* t, int64_t R, int32_t K, const double* T, int32_t theta,
               double dt, double gamma, uint64_t seed, int32_t mol, int32_t resample,
               int32_t n_threads, orc_obs* out, double* x, double* v, int32_t* fam, double* E) {
    int n = t->n_atoms;
    size_t rs = 3 * (size_t)n;
    double* x2 = (double*)malloc(sizeof(double) * rs * (size_t)R);
    double* v2 = (double*)malloc(sizeof(double) * rs * (size_t)R);
    int32_t* fam2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)R);
    double* E2 = (double*)malloc(sizeof(double) * (size_t)R);
    uint64_t* W = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)R);
    int32_t* cnt = (int32_t*)malloc(sizeof(int32_t) * (size_t)R);
    if (!x2 || !v2 || !fam2 || !E2 || !W || !cnt) return -1;

    uint32_t step = 0;
    double sum_lnq = 0.0;
    /* step 1: equilibrium ensemble at T0, plus theta steps for independence */
    orc_init(t, R, T[0], seed, mol, x, v, fam);
    orc_propagate(t, R, x, v, E, theta, dt, T[0], gamma, seed, step, mol, n_threads);
    step += (uint32_t)theta;
    memset(&out[0], 0, sizeof(orc_obs));
    orc_observables(t, R, x, v, fam, E, &out[0]);
    out[0].T = T[0];
    out[0].max_copies = 1;

    for (int32_t i = 1; i <= K; ++i) {
        /* step 2: resample to T_i with the relative Boltzmann weights */
        double lnq = orc_resample_weights(E, R, T[i - 1], T[i], W);
        if (resample) {
            orc_multinomial_counts(W, R, seed, (uint32_t)i, mol, cnt);
        } else {
            for (int64_t j = 0; j < R; ++j) cnt[j] = 1;
        }
        int32_t maxc = 0;
        for (int64_t j = 0; j < R; ++j) if (cnt[j] > maxc) maxc = cnt[j];
        orc_gather(t, R, cnt, x, v, fam, E, sqrt(T[i] / T[i - 1]), x2, v2, fam2, E2);
        memcpy(x, x2, sizeof(double) * rs * (size_t)R);
        memcpy(v, v2, sizeof(double) * rs * (size_t)R);
        memcpy(fam, fam2, sizeof(int32_t) * (size_t)R);
        sum_lnq += lnq;
        /* step 3: theta MD steps per copy at T_i */
        orc_propagate(t, R, x, v, E, theta, dt, T[i], gamma, seed, step, mol, n_threads);
        step += (uint32_t)theta;
        /* step 4: population averages at T_i */
        memset(&out[i], 0, sizeof(orc_obs));
        orc_observables(t, R, x, v, fam, E, &out[i]);
        out[i].T = T[i];
        out[i].lnQ = lnq;
        out[i].sum_lnQ = sum_lnq;
        out[i].max_copies = maxc;
    }
    free(x2); free(v2); free(fam2); free(E2); free(W); free(cnt);
    return 0;
}
