/*
 * pamd_oracle.h -- interface of the FP64 CPU oracle (test infrastructure).
 * Only the test suite, the smoke check and the benchmark's CPU legs use it.
 * It is unrelated to include/pamd.h, the CUDA library's interface.
 */
#ifndef PAMD_ORACLE_H
#define PAMD_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_PURPOSE_NOISE 0u
#define ORC_PURPOSE_INIT 1u
#define ORC_PURPOSE_RESAMPLE 2u
#define ORC_NBINS 64

typedef struct {
    int32_t n_atoms;
    const double *mass, *charge, *sigma, *epsilon, *x0; /* [N], x0 [N][3] */
    int32_t n_bonds;
    const int32_t* bond; /* [nb][2] */
    const double *bond_r0, *bond_k;
    int32_t n_angles;
    const int32_t* angle; /* [na][3] */
    const double *angle_t0, *angle_k;
    int32_t n_dihedrals;
    const int32_t* dihedral; /* [nd][4] */
    const int32_t* dih_n;
    const double *dih_k, *dih_phase;
    int32_t n_excl;
    const int32_t* excl; /* [ne][2] */
    int32_t n_pair14;
    const int32_t* pair14; /* [n14][2] */
    double scale14_lj, scale14_coul;
} orc_topology;

typedef struct {
    double T, lnQ, sum_lnQ;
    double e_pot, e_pot_se, e_kin, e_kin_se, t_meas;
    double rg, rg_se, rg2, rg2_se;
    int64_t n_families;
    int32_t max_copies;
    int32_t pad_;
} orc_obs;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_normal3(uint64_t seed, uint32_t atom, uint32_t slot, uint32_t step, uint32_t purpose,
                 double z[3]);
double orc_exp_det(double x);
double orc_dihedral_angle(const double* xi, const double* xj, const double* xk, const double* xl);
double orc_energy_forces(const orc_topology* t, const double* x, double* f, double* terms);
void orc_init(const orc_topology* t, int64_t R, double T0, uint64_t seed, int32_t mol, double* x,
              double* v, int32_t* fam);
void orc_propagate(const orc_topology* t, int64_t R, double* x, double* v, double* E,
                   int32_t theta, double dt, double T, double gamma, uint64_t seed,
                   uint32_t step0, int32_t mol, int32_t n_threads);
void orc_propagate_slots(const orc_topology* t, int64_t R, const int64_t* slots, double* x,
                         double* v, double* E, int32_t theta, double dt, double T, double gamma,
                         uint64_t seed, uint32_t step0, int32_t mol, int32_t n_threads);
void orc_energies(const orc_topology* t, int64_t R, const double* x, double* E);
int32_t orc_weight_shift(int64_t R);
double orc_resample_weights(const double* E, int64_t R, double T_prev, double T_next, uint64_t* W);
int64_t orc_ancestor(const uint64_t* C, int64_t R, uint64_t t);
uint64_t orc_resample_uniform(uint64_t seed, uint32_t k, uint32_t temp_index, int32_t mol);
void orc_multinomial_counts(const uint64_t* W, int64_t R, uint64_t seed, uint32_t temp_index,
                            int32_t mol, int32_t* counts);
void orc_gather(const orc_topology* t, int64_t R, const int32_t* counts, const double* x,
                const double* v, const int32_t* fam, const double* E, double vscale,
                double* x_new, double* v_new, int32_t* fam_new, double* E_new);
double orc_kinetic(const orc_topology* t, const double* v);
double orc_rgyr(const orc_topology* t, const double* x);
void orc_observables(const orc_topology* t, int64_t R, const double* x, const double* v,
                     const int32_t* fam, const double* E, orc_obs* o);
int orc_anneal(const orc_topology* t, int64_t R, int32_t K, const double* T, int32_t theta,
               double dt, double gamma, uint64_t seed, int32_t mol, int32_t resample,
               int32_t n_threads, orc_obs* out, double* x, double* v, int32_t* fam, double* E);

#ifdef __cplusplus
}
#endif
#endif
