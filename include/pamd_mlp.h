/*
 * pamd_mlp.h -- learned energy surrogate for population-annealing MD.
 *
 * The paper integrates every replica with an exact force field (Section 2:
 * each replica is advanced by theta MD steps at the current temperature).
 * This interface adds a learned alternative that stands beside it: a small
 * multilayer perceptron over inverse pair distances,
 *
 *   g_p  = 1 / r_ij for every pair p = (i, j), i < j, in row order
 *          (p = 0: (0,1), (0,2), ..., (0,N-1), then (1,2), ...),
 *          P = N (N - 1) / 2 pairs, normalised a_p = (g_p - mu_p) / sd_p;
 *   h1   = silu(W1 a + b1),  W1 [H][P];
 *   h2   = silu(W2 h1 + b2), W2 [H][H];
 *   e    = w3 . h2 + b3,     E = sigma_E e + mu_E   (kJ/mol);
 *   F_k  = -dE/dx_k         (kJ/mol/nm), by the analytic backward pass,
 *
 * with silu(z) = z / (1 + exp(-z)).  The dense layers run on the tensor
 * cores with BF16 operands (weights, normalised features, activations and
 * back-propagated signals are rounded to BF16) and FP32 accumulation; the
 * rest is FP32, the energy is returned in FP64.
 *
 * Training minimises, over a minibatch of M samples (positions x, reference
 * energies E_ref and forces F_ref, normally from exact PAMD runs),
 *
 *   L = (1/M) sum_m [ (e_m - e_ref,m)^2 + lam / (3N) sum_k |f_mk - f_ref,mk|^2 ],
 *   e_ref = (E_ref - mu_E) / sigma_E,  f = F / sigma_E,  f_ref = F_ref / sigma_E,
 *
 * whose gradient needs the derivative of the forces with respect to the
 * weights (a forward tangent pass and the reverse of it); every step runs in
 * this library's kernels.  Weights are updated by Adam (Kingma & Ba 2015).
 *
 * A model attached to a population (pamd_set_force_model) replaces the exact
 * forces and energies in pamd_propagate and pamd_anneal; the BAOAB update,
 * the noise stream and the resampling are unchanged.  Each MD step is one
 * step kernel and four GEMM launches; pamd_anneal captures the whole anneal
 * as one CUDA graph in which every temperature's theta steps are a
 * conditional WHILE node (the step index is kept in device memory), and
 * re-captures it when the model, its workspace or its energy scale changes.
 * The model must not be used from another stream while such an anneal runs.
 *
 * Memory layouts (all row-major, C order):
 *   positions, forces  [M][N][3] FP32 (nm, kJ/mol/nm) in device memory;
 *   energies           [M] FP64 (kJ/mol) in device memory;
 *   parameters         host FP32 arrays as in pamd_mlp_params.
 * Every call returns PAMD_OK (0) or a negative PAMD_* code from pamd.h with a
 * message for pamd_last_error(); a model whose kernels failed stays unusable
 * (PAMD_ESTATE).  Calls on one model are not thread-safe.
 */
#ifndef PAMD_MLP_H
#define PAMD_MLP_H

#include <stdint.h>

#include "pamd.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pamd_mlp pamd_mlp;

/* Host copies of the parameters (caller-owned arrays; P = N (N-1) / 2).
 * Used by pamd_mlp_set_params (read), pamd_mlp_get_params and
 * pamd_mlp_get_grads (written; for the gradient the normalisation members
 * are left untouched).  A NULL array is skipped. */
typedef struct pamd_mlp_params {
    float* W1;      /* [H][P] */
    float* b1;      /* [H] */
    float* W2;      /* [H][H] */
    float* b2;      /* [H] */
    float* w3;      /* [H] */
    double b3;
    float* mu;      /* [P] feature means */
    float* sd;      /* [P] feature standard deviations (> 0) */
    double mu_E;    /* energy offset (kJ/mol) */
    double sigma_E; /* energy scale (kJ/mol, > 0) */
} pamd_mlp_params;

/*
 * BF16 tensor-core matrix product (the building block of the dense layers):
 * C = A . B^T with A [M][lda], B [N][ldb] row-major __nv_bfloat16 in device
 * memory (only the first K columns read), C [M][ldc] FP32 in device memory,
 * FP32 accumulation.  K, lda and ldb must be multiples of 8, lda, ldb >= K,
 * ldc >= N, and A, B 16-byte aligned.  stream: cudaStream_t (NULL = legacy
 * default).  Synchronises the stream.  Errors: PAMD_EINVAL, PAMD_ECUDA,
 * PAMD_ETIMEOUT (the tensor-core pipeline did not finish).
 */
int pamd_gemm_bf16(const void* A, const void* B, float* C, int32_t M, int32_t N, int32_t K,
                   int32_t lda, int32_t ldb, int32_t ldc, void* stream);

/*
 * Device time of the product above: `reps` (1..1000) back-to-back launches
 * bracketed by two CUDA events recorded on `stream`; *ms_out receives the
 * mean time per launch in milliseconds and C the product.  Arguments and
 * errors as for pamd_gemm_bf16 (PAMD_EINVAL also for reps or a null ms_out).
 */
int pamd_gemm_bf16_time(const void* A, const void* B, float* C, int32_t M, int32_t N, int32_t K,
                        int32_t lda, int32_t ldb, int32_t ldc, int32_t reps, void* stream,
                        float* ms_out);

/*
 * New model for molecules of n_atoms atoms (2..PAMD_MAX_ATOMS) with hidden
 * width `hidden` (32..1024, a multiple of 32).  Weights are drawn from
 * N(0, 1/fan_in) by a Philox stream keyed on `seed`, biases are 0, mu = 0,
 * sd = 1, mu_E = 0, sigma_E = 1.  stream: cudaStream_t all of the model's
 * work is queued on (NULL: the library creates one).  Errors: PAMD_EINVAL,
 * PAMD_ENOMEM, PAMD_ECUDA.
 */
int pamd_mlp_create(pamd_mlp** out, int32_t n_atoms, int32_t hidden, uint64_t seed, void* stream);

/* Shape of a model: atoms, pairs P and hidden width. */
int pamd_mlp_info(pamd_mlp* mlp, int32_t* n_atoms, int32_t* n_pairs, int32_t* hidden);

/* Copy parameters in (set) or out (get); see pamd_mlp_params.  set resets
 * the Adam moments.  Synchronous. */
int pamd_mlp_set_params(pamd_mlp* mlp, const pamd_mlp_params* p);
int pamd_mlp_get_params(pamd_mlp* mlp, pamd_mlp_params* p);

/*
 * Set the normalisation from data: mu_p and sd_p as the mean and standard
 * deviation (population, n in the denominator) of g_p over the n
 * configurations x_dev [n][N][3], mu_E and sigma_E those of E_dev [n];
 * a zero standard deviation becomes 1.  Computed in FP64 on the GPU.
 * Synchronous.  Errors: PAMD_EINVAL (n < 2, null pointer), PAMD_ECUDA.
 */
int pamd_mlp_fit_normalization(pamd_mlp* mlp, const float* x_dev, const double* E_dev, int64_t n);

/*
 * Surrogate energies E_dev [M] (FP64, or NULL) and forces F_dev [M][N][3]
 * (FP32, or NULL) of the configurations x_dev [M][N][3].  Asynchronous on
 * the model's stream.  Errors: PAMD_EINVAL, PAMD_ENOMEM (workspace),
 * PAMD_ECUDA.
 */
int pamd_mlp_energy_forces(pamd_mlp* mlp, const float* x_dev, int64_t M, double* E_dev,
                           float* F_dev);

/*
 * Loss L of the minibatch (definition above) and its gradient with respect
 * to W1, b1, W2, b2, w3 and b3, kept in the model for pamd_mlp_get_grads and
 * pamd_mlp_adam_step.  The minibatch is samples idx_dev[0..M-1] (device
 * int32, or NULL for samples 0..M-1) of x_dev [n][N][3], E_dev [n] and
 * F_dev [n][N][3].  M: 4..65536, a multiple of 4.  lam >= 0 weights the
 * force term.  loss: host output (the call then synchronises), or NULL
 * (asynchronous).  Errors: PAMD_EINVAL, PAMD_ENOMEM, PAMD_ECUDA,
 * PAMD_ETIMEOUT.
 */
int pamd_mlp_loss_grads(pamd_mlp* mlp, const float* x_dev, const double* E_dev,
                        const float* F_dev, const int32_t* idx_dev, int64_t M, double lam,
                        double* loss);

/* Gradient of the last pamd_mlp_loss_grads call (synchronous). */
int pamd_mlp_get_grads(pamd_mlp* mlp, pamd_mlp_params* g);

/* One Adam update of the weights from the last gradient (step size lr,
 * moment decays beta1, beta2, denominator offset eps, bias-corrected).
 * Asynchronous. */
int pamd_mlp_adam_step(pamd_mlp* mlp, double lr, double beta1, double beta2, double eps);

/*
 * Use `mlp` (or, with NULL, the exact force field again) for the forces and
 * energies of every later pamd_propagate and pamd_anneal on ctx.  The model
 * must be for ctx's atom count, must outlive its use, and must not be
 * trained while attached.  Single-molecule mixed-precision contexts only
 * (PAMD_EUNSUPPORTED otherwise).  Allocates the model's workspace for ctx's
 * population.  Errors: PAMD_EINVAL, PAMD_EUNSUPPORTED, PAMD_ENOMEM.
 */
int pamd_set_force_model(pamd_ctx* ctx, pamd_mlp* mlp);

/*
 * Model files: pamd_mlp_save writes the shape and every parameter (FP32, the
 * normalisation included) with a checksum, in the machine's byte order, to
 * `path` (via path.tmp and a rename); pamd_mlp_load creates a model from such
 * a file (stream as in pamd_mlp_create).  Synchronous.  Errors: PAMD_EINVAL
 * (null argument, unreadable or unwritable file, not a model file, checksum
 * mismatch), PAMD_ENOMEM, PAMD_ECUDA.
 */
int pamd_mlp_save(pamd_mlp* mlp, const char* path);
int pamd_mlp_load(pamd_mlp** out, const char* path, void* stream);

/* Wait for the model's queued work; PAMD_ETIMEOUT if a tensor-core
 * pipeline wait ran out, PAMD_ECUDA on an asynchronous CUDA error. */
int pamd_mlp_sync(pamd_mlp* mlp);

/* Kernel launches the model issued so far. */
int64_t pamd_mlp_launch_count(pamd_mlp* mlp);

/* Free the model (NULL is allowed). */
void pamd_mlp_destroy(pamd_mlp* mlp);

#ifdef __cplusplus
}
#endif
#endif /* PAMD_MLP_H */
