/*
 * pamd_adaptive.h -- temperature schedules chosen from an overlap condition
 * (part of libpamd).
 *
 * The PAMD scheme of Christiansen, Weigel & Janke, arXiv:1806.06016, picks
 * its temperatures by the rules of parallel tempering (enough overlap of the
 * energy histograms of neighbouring temperatures) and notes that they can be
 * chosen automatically from an overlap condition.  The overlap of the
 * canonical energy distributions at T_prev and T < T_prev is estimated from
 * the population at T_prev (Barash et al. 2017): with potential energies
 * E_j, j < R, and dbeta = 1/(k_B T) - 1/(k_B T_prev),
 *     tau_j(dbeta) = R exp(-dbeta E_j) / sum_k exp(-dbeta E_k)
 *     alpha(dbeta) = (1/R) sum_j min(1, tau_j(dbeta)),
 * which is 1 at dbeta = 0 and falls as dbeta grows.  The next temperature is
 * T_final when alpha at T_final is at least alpha_target, and otherwise the
 * temperature where alpha equals alpha_target, found by a multisection
 * search on the GPU to about 1e-6 of dbeta_final (the exponentials in FP32
 * on E_j - min E, the sums in FP64).  The returned temperature always meets
 * the condition by the GPU's estimate.
 */
#ifndef PAMD_ADAPTIVE_H
#define PAMD_ADAPTIVE_H

#include "pamd.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Next temperature for R finite energies already on the device (E_dev [R]
 * FP64).  T_next_out: host double.  alpha_out: host double or NULL, the
 * estimated overlap at T_next.  Allocates its scratch stream-ordered
 * (cudaMallocAsync, about 4 R bytes) on stream (cudaStream_t, NULL = legacy
 * default) and synchronises it.  Errors: PAMD_EINVAL (null pointer, R < 1,
 * not 0 < T_final < T_prev, alpha_target outside (0, 1)), PAMD_ENONFINITE (a
 * non-finite energy), PAMD_ENOMEM, PAMD_ECUDA.
 */
int pamd_overlap_temperature(const double* E_dev, int64_t R, double T_prev, double T_final,
                             double alpha_target, double* T_next_out, double* alpha_out,
                             void* stream);

/*
 * The same for the context's current population (its energies after the
 * last propagate), with scratch owned by the context.  Synchronises.
 * Single-molecule contexts only.
 */
int pamd_next_temperature(pamd_ctx* ctx, double T_prev, double T_final, double alpha_target,
                          double* T_next_out, double* alpha_out);

/*
 * A whole anneal whose temperatures come from the overlap condition: theta
 * steps at T0, measure; then while T > T_final and fewer than max_steps
 * resamplings: choose T_next (pamd_next_temperature), resample T -> T_next
 * (resample = 0: the resampling-off control, copies all 1), theta steps at
 * T_next, measure.  obs_out: host [max_steps + 1] or NULL; T_out: host
 * [max_steps + 1] or NULL (the temperatures used); n_temps_out: host, the
 * number of temperatures measured (resamplings + 1).  Energies are recorded
 * as in pamd_anneal when pamd_record_energies is on (row i = i-th
 * temperature).  Issues the steps one by one (two synchronisations per
 * temperature), not as one graph.  Errors: as pamd_anneal, plus PAMD_EINVAL
 * for alpha_target outside (0, 1), T_final >= T0 or max_steps < 0, or when
 * a step cannot lower the temperature (the overlap falls below the target
 * within the search resolution); the population then stays at the last
 * temperature reached.
 */
int pamd_anneal_adaptive(pamd_ctx* ctx, double T0, double T_final, double alpha_target,
                         int32_t theta, double dt_ps, int32_t max_steps, int32_t resample,
                         pamd_obs* obs_out, double* T_out, int32_t* n_temps_out);

#ifdef __cplusplus
}
#endif

#endif /* PAMD_ADAPTIVE_H */
