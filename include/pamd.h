/*
 * pamd.h -- C interface of libpamd, a CUDA (sm_103a) implementation of the
 * data-parallel hot path of population-annealing molecular dynamics (PAMD),
 * Christiansen, Weigel & Janke, "Accelerating molecular dynamics simulations
 * with population annealing", arXiv:1806.06016.
 *
 * The calls follow the paper's statement of the method (the five-step PAMD
 * scheme): pamd_init sets up R copies of a molecule at T0 (step 1),
 * pamd_resample replicates each copy in proportion to its relative Boltzmann
 * weight and rescales velocities (step 2), pamd_propagate runs theta Langevin
 * MD steps per copy (step 3), and pamd_observables returns population
 * averages (step 4).  pamd_anneal runs steps 2-4 over a whole temperature
 * schedule as one CUDA graph.
 *
 * Units: nm, ps, amu, elementary charge, K, kJ/mol.  k_B = 0.008314462618
 * kJ/mol/K, Coulomb constant 138.935458 kJ mol^-1 nm e^-2.
 *
 * Conventions for every function below:
 *   - The return value is PAMD_OK (0) or a negative PAMD_E* code; a
 *     thread-local message is available from pamd_last_error().  No call
 *     aborts or exits the process.
 *   - On an argument error the context is left unchanged.  If a CUDA call
 *     fails part-way the context is marked broken and every later call except
 *     pamd_destroy returns PAMD_ESTATE.
 *   - Host pointers are caller-owned and only read/written during the call.
 *     Device memory is owned by the context and obtained from
 *     pamd_options.dev_alloc (cudaMalloc when NULL).
 *   - Work is issued on pamd_options.stream.  Calls that return host data
 *     synchronise that stream; pamd_propagate and pamd_resample with NULL
 *     host outputs return without synchronising.
 *   - The library keeps all replica state on the device in FP32 (positions
 *     relative to the molecule's centre of mass, velocities) with FP64
 *     potential energies, weights, ln Q and the free-energy sum.
 */
#ifndef PAMD_H
#define PAMD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PAMD_OK 0
#define PAMD_EINVAL (-1)      /* bad argument (null pointer, size, index, range) */
#define PAMD_ENOMEM (-2)      /* device or host allocation failed */
#define PAMD_ECUDA (-3)       /* a CUDA runtime call failed */
#define PAMD_ETIMEOUT (-4)    /* a bounded device-side wait gave up */
#define PAMD_ENONFINITE (-5)  /* a replica's energy became NaN or infinite */
#define PAMD_ESTATE (-6)      /* the context is broken by an earlier failure */
#define PAMD_EUNSUPPORTED (-7) /* valid request the library cannot serve */
#define PAMD_EPOPSIZE (-8)    /* a variable-size resampling left the population empty or above its capacity */

/* Largest molecule the shared-memory kernels hold (atoms). */
#define PAMD_MAX_ATOMS 256

#define PAMD_PREC_MIXED 0 /* FP32 forces/integration, FP64 energies and weights */
#define PAMD_PREC_FP64 1  /* everything in FP64 on the GPU */

/*
 * Resampling rules (the resampling paragraph: the paper draws R multinomial
 * samples and notes that other implementations exist).  Both keep the
 * population size R and use the same integer weights W_j and inclusive sums
 * C_j (C = C_{R-1}); they differ in the targets t_k whose ancestor is the
 * first j with C_j > t_k:
 *   MULTINOMIAL  t_k = floor(u_k C / 2^64), u_k an independent 64-bit Philox
 *                uniform per new slot k;
 *   SYSTEMATIC   t_k = floor((k C + V) / R), V = floor(u_0 C / 2^64): one
 *                uniform per resampling, each n_j = floor(R W_j / C) or one
 *                more (lower variance of the copy numbers).
 */
#define PAMD_RESAMPLE_MULTINOMIAL 0
#define PAMD_RESAMPLE_SYSTEMATIC 1
/*
 * Two more rules let the population size fluctuate around the target R
 * given to pamd_init (Wang, Machta & Katzgraber 2015): copy numbers with
 * E[n_j] = tau_j = R W_j / C, the same integer weights, C their sum over the
 * live population:
 *   NEAREST  n_j = floor(tau_j), plus one with probability frac(tau_j) (the
 *            64-bit Philox uniform u_j of ancestor j: one more copy when
 *            floor(u_j C / 2^64) < R W_j - C floor(tau_j), exact integers);
 *   POISSON  n_j ~ Poisson(tau_j): lambda = (double(R) double(W_j)) / double(C)
 *            split into m = ceil(lambda / 500) chunks, each drawn by FP64
 *            inversion of the Poisson CDF with the uniform of Philox counter
 *            (j, resampling index, chunk, 2 | mol << 8).
 * ln Q stays ln((1/R~) sum_j w_j) over the live size R~.  The context then
 * holds a capacity of R + 8 ceil(sqrt(R)) + 64 slots (pamd_info reports the
 * capacity as R; pamd_population_size the live size); the live replicas are
 * the first slots.  Mixed precision, exact forces, one replica per lane
 * group, single-molecule contexts only; pamd_record_energies, the adaptive
 * schedule and checkpoint files are not available with them.
 */
#define PAMD_RESAMPLE_NEAREST 2
#define PAMD_RESAMPLE_POISSON 3

typedef struct pamd_ctx pamd_ctx; /* opaque, owned by the library */

/*
 * Force field of one molecule (test-system paragraph: a peptide in vacuo,
 * all pairs, no cutoff).  Arrays are read during pamd_init only.
 *   bonds      E = 1/2 k (r - r0)^2                (pairs [n][2])
 *   angles     E = 1/2 k (theta - theta0)^2        (triples [n][3], rad)
 *   dihedrals  E = k (1 + cos(n phi - phase))      (quadruples [n][4], n in 1..6)
 *   nonbonded  for every pair not in excl: LJ 4 eps [(sig/r)^12 - (sig/r)^6]
 *              with sig = (sig_i + sig_j)/2, eps = sqrt(eps_i eps_j), plus
 *              Coulomb k_e q_i q_j / r; pairs listed in pair14 are scaled by
 *              scale14_lj and scale14_coul.  A pair in both lists is excluded.
 */
typedef struct pamd_topology {
    int32_t n_atoms;          /* 1 .. PAMD_MAX_ATOMS */
    const double* mass;       /* [N] amu, > 0 */
    const double* charge;     /* [N] e */
    const double* sigma;      /* [N] nm, >= 0 */
    const double* epsilon;    /* [N] kJ/mol, >= 0 */
    const double* x0;         /* [N][3] nm, start geometry */
    int32_t n_bonds;
    const int32_t* bond;      /* [n_bonds][2] */
    const double* bond_r0;    /* [n_bonds] nm */
    const double* bond_k;     /* [n_bonds] kJ/mol/nm^2 */
    int32_t n_angles;
    const int32_t* angle;     /* [n_angles][3], vertex in the middle */
    const double* angle_t0;   /* [n_angles] rad */
    const double* angle_k;    /* [n_angles] kJ/mol/rad^2 */
    int32_t n_dihedrals;
    const int32_t* dihedral;  /* [n_dihedrals][4] */
    const int32_t* dih_n;     /* [n_dihedrals] multiplicity 1..6 */
    const double* dih_k;      /* [n_dihedrals] kJ/mol */
    const double* dih_phase;  /* [n_dihedrals] rad */
    int32_t n_excl;
    const int32_t* excl;      /* [n_excl][2] pairs left out of the nonbonded sum */
    int32_t n_pair14;
    const int32_t* pair14;    /* [n_pair14][2] pairs with scaled nonbonded terms */
    double scale14_lj;
    double scale14_coul;
} pamd_topology;

typedef struct pamd_options {
    double gamma_per_ps;        /* Langevin friction (MD-parameters paragraph: 1/ps) */
    int32_t precision;          /* PAMD_PREC_MIXED or PAMD_PREC_FP64 */
    int32_t lanes_per_replica;  /* 0 = choose; else 1..32 lanes, with at most 8 atoms
                                   per lane (ceil(n_atoms / lanes) <= 8) */
    int32_t warps_per_block;    /* 0 = choose (4); else 1..8, lowered to the kernel's
                                   block-size cap (4 warps for the packed-pair kernel
                                   and for 5 atoms per lane) and to shared memory */
    int32_t mol_id;             /* molecule index mixed into the random counters */
    int32_t autotune;           /* 1: pamd_autotune(ctx, 20, NULL) at the end of pamd_init */
    int32_t replicas_per_lane;  /* 0 or 1: one replica per lane group; 2: two replicas per
                                   group in packed FP32x2 arithmetic (2..4 atoms per lane) */
    void* (*dev_alloc)(size_t bytes, void* user); /* NULL = cudaMalloc */
    void (*dev_free)(void* ptr, void* user);      /* NULL = cudaFree */
    void* alloc_user;
    void* stream;               /* cudaStream_t; NULL = a non-blocking stream the context creates */
    int32_t resample_rule;      /* PAMD_RESAMPLE_MULTINOMIAL (the paper's choice) or
                                   PAMD_RESAMPLE_SYSTEMATIC */
    int32_t pair_arith;         /* PAMD_PAIRS_AUTO (0), PAMD_PAIRS_SCALAR or PAMD_PAIRS_PACKED */
} pamd_options;

/* Arithmetic of the nonbonded pair loop (pamd_options.pair_arith).  PACKED
 * holds each lane's own atoms in register pairs and evaluates two pairs per
 * add/mul/fma.f32x2 instruction (same FP32 roundings as the scalar form);
 * linear chains with 3..8 atoms per lane and one replica per lane group
 * only.  AUTO starts with PACKED where it applies (mixed precision, one
 * replica per lane group), else SCALAR; pamd_autotune times both where
 * PACKED applies and keeps the faster. */
#define PAMD_PAIRS_AUTO 0
#define PAMD_PAIRS_SCALAR 1
#define PAMD_PAIRS_PACKED 2

/* Per-temperature population averages (PAMD scheme, step 4) with jackknife
 * errors over 64 family bins (paragraph on correlations after resampling). */
typedef struct pamd_obs {
    double T;          /* heat-bath temperature of this measurement */
    double lnQ;        /* ln Q of the resampling that led here (0 at T0) */
    double sum_lnQ;    /* sum of ln Q since T0 = ln Z(T) - ln Z(T0), configurational */
    double e_pot, e_pot_se;
    double e_kin, e_kin_se;
    double t_meas;     /* 2 <E_kin> / (3 N k_B) */
    double rg, rg_se;  /* radius of gyration sqrt(mean |x_i - xbar|^2) */
    double rg2, rg2_se;
    int64_t n_families; /* distinct family ids (ancestors at T0) alive */
    int32_t max_copies; /* largest copy count of the resampling that led here */
    int32_t pad_;
    int64_t R_live;     /* population size at this measurement */
} pamd_obs;

/* Fill *opt with the defaults: gamma 1/ps, mixed precision, automatic
 * launch shape, molecule 0, cudaMalloc/cudaFree, a stream of the context's own. */
void pamd_options_default(pamd_options* opt);

/*
 * PAMD scheme, step 1.  Create a context holding R replicas of `top`: every
 * replica starts from x0 (shifted to its centre of mass), velocities from the
 * Maxwell-Boltzmann distribution at T0 drawn from Philox4x32-10 keyed on
 * `seed`, family id = replica index.  The random counter layout is
 * (atom, replica slot, step, purpose | mol_id << 8).
 * The paper's "additionally apply theta MD steps" is the caller's first
 * pamd_propagate at T0.
 * out: receives the context.  R: 1 .. 2^31-1.  T0 > 0.  opt: NULL = defaults.
 * Errors: PAMD_EINVAL (bad topology, R, T0), PAMD_ENOMEM, PAMD_ECUDA,
 * PAMD_EUNSUPPORTED (n_atoms > PAMD_MAX_ATOMS).
 */
int pamd_init(pamd_ctx** out, const pamd_topology* top, int64_t R, double T0, uint64_t seed,
              const pamd_options* opt);

/*
 * Batched independent anneals: n_mol molecules (1..64) of uneven size, each
 * with its own population R[m], start temperature T0[m] and Philox stream
 * (molecule index m mixed into the counters).  pamd_propagate advances them
 * all with one persistent launch per group of molecules sharing an
 * atoms-per-lane count (3..7) and pair arithmetic (a kernel compiled for
 * each, so that each group gets its own register allocation); the group
 * launches run concurrently on streams forked from the context's stream,
 * each taking (molecule, replica batch) items from its own device work queue,
 * largest molecules first.  A molecule whose topology is a linear chain
 * takes the packed FP32x2 pair arithmetic unless opt->pair_arith is
 * PAMD_PAIRS_SCALAR; other molecules take the scalar one.  On a batch context pamd_reset,
 * pamd_propagate, pamd_resample (copies_out: [sum R] in molecule order, lnQ_out:
 * [n_mol]), pamd_observables (out: [n_mol]) and pamd_anneal (per_step_out:
 * [(K+1) * n_mol], temperature-major; one CUDA graph for the whole batch) act
 * on every molecule with a common temperature schedule; state access goes
 * through pamd_batch_sub.  Mixed precision only.  opt: as for pamd_init
 * (lanes_per_replica, warps_per_block, mol_id and autotune are chosen per
 * molecule and ignored).
 */
int pamd_init_batch(pamd_ctx** out, int32_t n_mol, const pamd_topology* tops, const int64_t* R,
                    const double* T0, uint64_t seed, const pamd_options* opt);

/* Number of molecules of a batch context (0 for an ordinary context). */
int32_t pamd_batch_size(pamd_ctx* ctx);

/* The ordinary context of molecule m of a batch (owned by the batch: valid
 * until pamd_destroy of the batch, not to be destroyed separately), or NULL. */
pamd_ctx* pamd_batch_sub(pamd_ctx* ctx, int32_t m);

/*
 * PAMD scheme, step 1 again on an existing context: the population is reset
 * exactly as pamd_init left it for (T0, seed) -- start geometry, fresh
 * Maxwell-Boltzmann velocities, family id = slot -- and the random counters
 * and the running sum of ln Q return to zero.  No memory is allocated.
 * Asynchronous on the context's stream.
 */
int pamd_reset(pamd_ctx* ctx, double T0, uint64_t seed);

/*
 * PAMD scheme, step 3.  theta BAOAB Langevin steps (B: v += dt/2 F/m,
 * A: x += dt/2 v, O: v = c1 v + sqrt((1-c1^2) k_B T/m) xi, A, F(x), B;
 * c1 = exp(-gamma dt)) for every replica, one persistent kernel launch with
 * each replica held in shared memory for all theta steps.  Noise xi from
 * Philox keyed on (seed; atom, slot, global step, 0 | mol << 8).  Afterwards
 * the potential energy (FP64 sum of FP32 terms), kinetic energy and radius
 * of gyration of every replica are stored on the device.  Velocities are not
 * rescaled here.  theta >= 0 (0 only evaluates energies); dt_ps > 0; T > 0.
 * Asynchronous on the context's stream.
 */
int pamd_propagate(pamd_ctx* ctx, int32_t theta, double dt_ps, double T);

/*
 * PAMD scheme, step 2.  Resample from T_prev to T_next with the relative
 * Boltzmann weights tau_j = exp(-(beta_next - beta_prev) E_j) / Q,
 * Q = (1/R) sum_j exp(-(beta_next - beta_prev) E_j), by R multinomial draws
 * (paragraph on the resampling implementation: probabilities tau_j / R,
 * population size constant, zero copies prune).  Realisation: integer
 * weights W_j = floor(2^s exp(a_j - max a)), s = 63 - ceil(log2 R), inclusive
 * prefix sum C, draw k targets floor(u_k C_total / 2^64) with u_k a 64-bit
 * Philox uniform keyed on (slot k, resampling index, 0, 2 | mol << 8), and
 * ancestor = first j with C_j > target.  The new population lists copies in
 * ascending ancestor order; positions are recentred on the centre of mass,
 * velocities scaled by sqrt(T_next / T_prev), family ids carried along.
 * The running sum of ln Q is updated on the device.
 * copies_out: host [R] int32 copy counts n_j by ancestor, or NULL.
 * lnQ_out: host double, or NULL.  Either non-NULL synchronises the stream.
 */
int pamd_resample(pamd_ctx* ctx, double T_prev, double T_next, int32_t* copies_out,
                  double* lnQ_out);

/*
 * PAMD scheme, step 4.  Population averages of the current population
 * measured at temperature T (only recorded in out->T and t_meas is computed
 * from velocities).  out->lnQ / sum_lnQ / max_copies refer to the last
 * resampling.  Synchronises the stream.  Returns PAMD_ENONFINITE if any
 * replica energy is not finite.
 */
int pamd_observables(pamd_ctx* ctx, double T, pamd_obs* out);

/*
 * Whole anneal (PAMD scheme, steps 2-5 after the initial block): theta steps
 * at T[0], measure; then for i = 1..K: resample T[i-1] -> T[i] (or, with
 * resample = 0, keep every copy once and only rescale velocities: the
 * "anneal" control of the paper's Fig. 2), theta steps at T[i], measure.
 * Captured once per (K, theta, dt, schedule) into a CUDA graph and launched
 * as one graph.  per_step_out: host [K+1] or NULL.  Synchronises the stream.
 */
int pamd_anneal(pamd_ctx* ctx, int32_t K, const double* T, int32_t theta, double dt_ps,
                int32_t resample, pamd_obs* per_step_out);

/*
 * Copy the population to the host.  x, v: [R][N][3] double (the FP32 device
 * values widened), E: [R], fam: [R]; any may be NULL.  Synchronises.
 */
int pamd_get_state(pamd_ctx* ctx, double* x, double* v, double* E, int32_t* fam);

/*
 * Replace the population from the host.  x, v: [R][N][3] (rounded to FP32;
 * positions are stored as given, the caller recentres if it wants), E: [R]
 * or NULL (then left unchanged), fam: [R] or NULL (unchanged).
 */
int pamd_set_state(pamd_ctx* ctx, const double* x, const double* v, const double* E,
                   const int32_t* fam);

/*
 * Forces and potential energies of the current population without moving it
 * (the force evaluation of pamd_propagate, theta = 0).  f: host [R][N][3]
 * kJ/mol/nm or NULL; E: host [R] or NULL.  Synchronises.
 */
int pamd_forces(pamd_ctx* ctx, double* f, double* E);

/* Launch shape of the propagate kernel. */
typedef struct pamd_tune {
    int32_t lanes_per_replica; /* L: lanes of one warp that share a replica */
    int32_t atoms_per_lane;    /* B: atoms each lane owns */
    int32_t warps_per_block;
    int32_t replicas_per_lane; /* 1, or 2 for the packed two-replica kernels */
    int32_t from_cache;        /* 1 if the shape came from the cache */
    double ms;                 /* probe time of the chosen shape (0 if cached) */
    int32_t pair_arith;        /* PAMD_PAIRS_SCALAR or PAMD_PAIRS_PACKED */
    int32_t pad_;
} pamd_tune;

/*
 * Launch-shape autotuner (no counterpart in the paper; it picks how the
 * replica-parallel work of step 3 maps onto the GPU).  For every feasible
 * shape -- B = 1..8 atoms per lane with L = ceil(N/B) <= 32 lanes per replica
 * (fixed to the requested lanes_per_replica if one was given), one or two
 * replicas per lane group (two only for B = 2..4), and 2, 4 or 8 warps per
 * block -- one propagate launch of theta_probe steps over the whole
 * population is timed on a scratch copy; the fastest shape is kept.  The
 * population, energies, counters and observables are left unchanged.  The
 * choice is cached in the process per (N, R, chain layout) and, when the
 * environment variable PAMD_TUNE_CACHE names a file, in that file.
 * theta_probe: 1..1000.  out: chosen shape, or NULL.  Synchronises the
 * stream; must not be called while the stream is being captured.
 */
int pamd_autotune(pamd_ctx* ctx, int32_t theta_probe, pamd_tune* out);

/*
 * Copy counts and ln Q of one resampling, allocating no memory.  The paper
 * has no counterpart: this is a service for callers that cannot allocate
 * device memory -- code running under a framework that owns the whole device
 * pool (a custom operator whose memory must come from the host framework),
 * code that must not trigger the device-wide synchronisation cudaFree can
 * cause, or a loop with a fixed, pre-reserved memory budget.
 *
 * Computes exactly what pamd_resample computes for copies_out and lnQ_out
 * (same integer weights, prefix sums, Philox targets and ancestors; copy
 * counts identical bit for bit) from R energies already on the device, but
 * does not gather a population.  E_dev: device [R] FP64 potential energies.
 * resample_index and mol_id select the Philox stream as in pamd_resample (its
 * k-th call on a context uses index k).  counts_dev: device [R] int32 output,
 * n_j by ancestor.  lnQ_dev: device double output or NULL.  status_dev:
 * device int32 output or NULL; it receives 0, or PAMD_ENONFINITE when some
 * energy was NaN or infinite.  Such replicas get weight 0 (pamd_resample
 * reports the same case as PAMD_ENONFINITE); if every energy is non-finite
 * the counts are meaningless and ln Q is NaN, so a caller that cannot rule
 * this out must check status_dev.  stream: cudaStream_t (NULL = legacy
 * default).  Asynchronous: returns after queuing the work.
 *
 * Its scratch is one static device array of 2.1 MiB inside the library,
 * which every GPU that loads the library holds until the process exits; R
 * is therefore limited to 262144 (PAMD_EINVAL above).  No cudaMalloc, cudaFree
 * or allocating library routine is called.  Every call made outside stream
 * capture looks up the array's device address on the current device
 * (cudaGetSymbolAddress); a call on a stream that is being captured reuses the
 * address of that device's last uncaptured call, so the first call on a
 * device must come before any stream capture.  All calls share the array:
 * calls that overlap on the GPU (different streams, or different host threads
 * on one device) race with each other and must be serialised by the caller.
 * Errors: PAMD_EINVAL (null pointer, R, temperatures, mol_id), PAMD_ECUDA.
 */
int pamd_resample_counts_noalloc(const double* E_dev, int64_t R, double T_prev, double T_next,
                                 uint64_t seed, uint32_t resample_index, int32_t mol_id,
                                 int32_t* counts_dev, double* lnQ_dev, int32_t* status_dev,
                                 void* stream);

/*
 * Checkpoint files.  pamd_checkpoint writes the current population (state,
 * energies, family ids), the random-counter state (seed, MD step, resampling
 * index) and the running sum of ln Q to `path` (written to path.tmp, then
 * renamed), with a checksum.  pamd_restore reads such a file into a context
 * made for the same topology, population size and precision; afterwards the
 * run continues bit-identically to the one that wrote it.  The file is in
 * the machine's byte order.  A batch context is checkpointed molecule by
 * molecule (pamd_batch_sub).  Synchronous.  Errors: PAMD_EINVAL (null path,
 * unreadable or unwritable file, wrong magic, another population, checksum
 * mismatch; the context is unchanged), PAMD_EUNSUPPORTED (batch context),
 * PAMD_ECUDA.
 */
int pamd_checkpoint(pamd_ctx* ctx, const char* path);
int pamd_restore(pamd_ctx* ctx, const char* path);

/* Random-counter state: global MD step and resampling index.  A restarted
 * run that restores both (with the same seed and population) continues
 * bit-identically. */
int pamd_get_counters(pamd_ctx* ctx, uint32_t* step, uint32_t* resample_index, double* sum_lnQ);
int pamd_set_counters(pamd_ctx* ctx, uint32_t step, uint32_t resample_index, double sum_lnQ);

/* Number of replicas and atoms; the launch shape in use for propagate. */
int pamd_info(pamd_ctx* ctx, int64_t* R, int32_t* n_atoms, int32_t* lanes_per_replica,
              int32_t* atoms_per_lane, int32_t* replicas_per_block);

/* Live population size and capacity (slots of the population buffers); they
 * differ only under the NEAREST and POISSON resampling rules.  Synchronises
 * the context's stream.  Errors: PAMD_EINVAL (null context, batch context). */
int pamd_population_size(pamd_ctx* ctx, int64_t* live, int64_t* capacity);

/* Launch shape the propagate kernel of this context uses now (no
 * counterpart in the paper).  out->from_cache and out->ms are 0.  Errors:
 * PAMD_EINVAL (null argument, batch context). */
int pamd_get_shape(pamd_ctx* ctx, pamd_tune* out);

/* Number of kernel launches the library issued on this context so far. */
int64_t pamd_launch_count(pamd_ctx* ctx);

/* Wait for all work of the context; returns PAMD_ECUDA on an asynchronous
 * CUDA error. */
int pamd_sync(pamd_ctx* ctx);

/* Free the context and its device memory (NULL is allowed). */
void pamd_destroy(pamd_ctx* ctx);

/* Message of the last failing call on this thread ("" if none). */
const char* pamd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PAMD_H */
