/*
 * pamd_wham.h -- multiple-histogram reweighting (WHAM) of the potential
 * energies an anneal samples, on the GPU (part of libpamd).
 *
 * Free-energy paragraph of Christiansen, Weigel & Janke, arXiv:1806.06016:
 * the normalisation factors Q recorded at every resampling estimate ratios
 * of configurational partition functions, so their running sum gives
 * ln Z(T_i) - ln Z(T_0); those values start a few sweeps of the
 * self-consistency equations of the multiple-histogram method (Ferrenberg &
 * Swendsen 1989; Kumar et al. 1992), which refine ln Z(T_i) and give
 * reweighted averages at any temperature.
 *
 * Definitions.  Samples E[i][k], k < R, at T[i], i = 0..n_temps-1, beta_i =
 * 1 / (k_B T_i).  Histograms H_i(b) on n_bins equal bins over [e_min, e_max]
 * (width w = (e_max - e_min) / n_bins, centres E_b = e_min + (b + 1/2) w): a
 * sample goes to bin floor((E - e_min) * (n_bins / (e_max - e_min))), the top
 * edge to the last bin; samples outside the range or not finite are dropped
 * and N_i counts those kept.  H(b) = sum_i H_i(b).  One sweep computes
 *     g_b  = H(b) / sum_i N_i exp(-beta_i E_b - ln Z_i)
 *     Z_i  = sum_b g_b exp(-beta_i E_b)
 * and then restores the gauge ln Z_0 = 0; the sweeps stop after max_iter or
 * once the largest change of an ln Z_i in a sweep is below tol.  Sums of
 * exponentials are evaluated as max + ln sum exp(x - max), all in FP64.
 * Reweighted to T:  ln Z(T) = ln sum_b g_b exp(-E_b / k_B T), <E>(T) and
 * var E(T) = <(E - <E>)^2> under p_b = g_b exp(-E_b / k_B T) / Z(T).
 * Units: kJ/mol, K.
 */
#ifndef PAMD_WHAM_H
#define PAMD_WHAM_H

#include "pamd.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Record the potential energies pamd_anneal measures: after the theta steps
 * at T[i] (i = 0..K) the R energies of the population are copied to row i of
 * E_dev while i < rows.  E_dev: device memory, [rows][R] FP64, owned by the
 * caller and kept alive while recording is on; rows = 0 (E_dev may then be
 * NULL) turns recording off.  The copies are part of the anneal's CUDA graph
 * (a change of E_dev or rows re-captures it).  Single-molecule contexts only.
 * Errors: PAMD_EINVAL (batch context, rows < 0, E_dev NULL with rows > 0),
 * PAMD_ESTATE.
 */
int pamd_record_energies(pamd_ctx* ctx, double* E_dev, int32_t rows);

typedef struct pamd_wham_args {
    const double* E;        /* device [n_temps][R] energies (kJ/mol), row i sampled at T[i] */
    int32_t n_temps;        /* >= 1 */
    int64_t R;              /* samples per temperature, 1 .. 2^32 - 1 (32-bit bin counters) */
    const double* T;        /* host [n_temps] K, > 0 */
    int32_t n_bins;         /* 1 .. 65536 */
    double e_min, e_max;    /* histogram range; e_max <= e_min: [min E, max E] over the
                               finite samples, [min E, min E + 1] if they are all equal */
    const double* lnZ_init; /* host [n_temps] start values (e.g. the running sum of ln Q),
                               or NULL for zeros; shifted so that lnZ_init[0] = 0 */
    int32_t max_iter;       /* sweeps, >= 0 */
    double tol;             /* stop when the largest change of a sweep is below tol (0: never) */
    int32_t n_eval;         /* temperatures to reweight to, >= 0 */
    const double* T_eval;   /* host [n_eval] K, > 0 */
    void* stream;           /* cudaStream_t, NULL = legacy default stream */
} pamd_wham_args;

typedef struct pamd_wham_result {
    double* lnZ;            /* host [n_temps] out: ln Z(T_i) - ln Z(T_0) */
    double* ln_g;           /* host [n_bins] out or NULL: ln g_b, -inf for empty bins */
    uint32_t* hist;         /* host [n_temps][n_bins] out or NULL: the histograms */
    double* lnZ_eval;       /* host [n_eval] out or NULL: ln Z(T) in the same gauge */
    double* e_mean_eval;    /* host [n_eval] out or NULL: <E>(T) */
    double* e_var_eval;     /* host [n_eval] out or NULL: var E(T) */
    double e_min, bin_width;  /* out: the range used */
    int32_t iterations;     /* out: sweeps done */
    double max_delta;       /* out: largest change of ln Z in the last sweep (inf if none) */
} pamd_wham_result;

/*
 * Histograms and the self-consistency sweeps on the device (arguments and
 * definitions above).  Allocates its device workspace with cudaMalloc and
 * frees it before returning; synchronises the stream.  Deterministic: the
 * histograms use integer atomics, every floating-point sum a fixed order.
 * Errors: PAMD_EINVAL (null pointer, sizes, temperatures, no sample inside
 * the range), PAMD_ENOMEM, PAMD_ECUDA.
 */
int pamd_wham(const pamd_wham_args* args, pamd_wham_result* result);

#ifdef __cplusplus
}
#endif

#endif /* PAMD_WHAM_H */
