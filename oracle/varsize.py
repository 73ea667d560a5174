"""FP64 / exact-integer CPU oracle of the resampling rules that change the
population size -- TEST INFRASTRUCTURE.

Only the test suite and the benchmark's CPU legs use this module.  Plain
Python integers and numpy, written from the definitions below; Philox, the
deterministic exponential, the gather and the observables are the C oracle's
own (oracle/__init__.py).  Nothing is shared with the CUDA library.

The resampling paragraph of the paper draws R multinomial samples and notes
that other implementations of the step exist.  Two of them let the population
size fluctuate around a target R_t (Wang, Machta & Katzgraber 2015):

  nearest integer   n_j = floor(tau_j) + 1 with probability frac(tau_j),
                    else floor(tau_j);
  Poisson           n_j ~ Poisson(tau_j).

Both have E[n_j] = tau_j.  Here tau_j is normalised to the target size,
tau_j = R_t w_j / sum_k w_k with w_j = exp(-(beta_next - beta_prev) E_j), so
that E[sum_j n_j] = R_t whatever the current size R~ is.  The free-energy
increment keeps its definition over the current population,
ln Q = ln((1/R~) sum_j w_j).

Realisation (readings of the paper's silence, exact and deterministic so that
the GPU can be compared bit for bit):
  * the weights are the multinomial's integer weights W_j = floor(2^s
    exp_det(a_j - max a)), s = 63 - ceil(log2 R~), C = sum_j W_j, so that
    tau_j = R_t W_j / C is an exact rational;
  * nearest integer: q_j = floor(R_t W_j / C), r_j = R_t W_j - q_j C, and one
    more copy when floor(u_j C / 2^64) < r_j, u_j the 64-bit Philox uniform of
    ancestor j (counter (j, resampling index, 0, RESAMPLE | mol << 8), the
    multinomial's uniform for slot j): probability r_j / C = frac(tau_j) up
    to 2^-64;
  * Poisson: lambda_j = (double(R_t) * double(W_j)) / double(C) in FP64,
    split into m = ceil(lambda_j / 500) equal chunks lambda_j / m (so that
    e^-chunk stays far above the FP64 underflow); each chunk c is drawn by
    inversion of the Poisson CDF with u = (floor(u64 / 2^11) + 1/2) 2^-53, u64
    the Philox output of counter (j, resampling index, c, RESAMPLE | mol << 8):
    p_0 = exp_det(-lambda), F = p_0, n = 0; while u > F and n < n_max:
    n += 1, p = (p lambda) / n, F = F + p; n_max = floor(lambda + 20
    sqrt(lambda)) + 50.  n_j is the sum over the chunks.
"""
from __future__ import annotations

import math

import numpy as np

import oracle as _orc

CHUNK = 500.0


def _u64(seed, k, temp_index, word2, mol):
    o = _orc.philox4x32_10([k & 0xffffffff, temp_index & 0xffffffff, word2 & 0xffffffff,
                            _orc.PURPOSE_RESAMPLE | (mol << 8)],
                           [seed & 0xffffffff, (seed >> 32) & 0xffffffff])
    return int(o[0]) | (int(o[1]) << 32)


def nearest_integer_counts(W, R_target, seed, temp_index, mol=0):
    """Copy counts n_j (int32) of nearest-integer resampling."""
    W = [int(w) for w in np.asarray(W, dtype=np.uint64)]
    C = sum(W)
    cnt = np.zeros(len(W), np.int64)
    for j, w in enumerate(W):
        q, r = divmod(R_target * w, C)
        u = _u64(seed, j, temp_index, 0, mol)
        cnt[j] = q + (1 if ((u * C) >> 64) < r else 0)
    return cnt.astype(np.int32)


def poisson_inverse(lam, u):
    """Smallest n with F(n) >= u for the Poisson CDF F of mean lam (FP64, the
    summation order of the definition above)."""
    n_max = int(math.floor(lam + 20.0 * math.sqrt(lam))) + 50
    p = float(_orc.exp_det(-lam))
    F = p
    n = 0
    while u > F and n < n_max:
        n += 1
        p = (p * lam) / float(n)
        F = F + p
    return n


def poisson_counts(W, R_target, seed, temp_index, mol=0):
    """Copy counts n_j (int32) of Poisson resampling."""
    W = [int(w) for w in np.asarray(W, dtype=np.uint64)]
    C = sum(W)
    Cd = float(C)
    cnt = np.zeros(len(W), np.int64)
    for j, w in enumerate(W):
        lam = (float(R_target) * float(w)) / Cd
        m = max(1, int(math.ceil(lam / CHUNK)))
        chunk = lam / float(m)
        n = 0
        for c in range(m):
            u64 = _u64(seed, j, temp_index, c, mol)
            u = (float(u64 >> 11) + 0.5) * 2.0 ** -53
            n += poisson_inverse(chunk, u)
        cnt[j] = n
    return cnt.astype(np.int32)


def gather(top, counts, x, v, fam, E, vscale):
    """New population of sum(counts) replicas in ascending ancestor order:
    positions recentred, velocities scaled, family ids and energies carried
    (the C oracle's gather, with outputs sized for the new population)."""
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    n_new = int(counts.sum())
    t = _orc._topo(top)
    x = _orc._f64(x); v = _orc._f64(v); E = _orc._f64(E)
    fam = np.ascontiguousarray(fam, dtype=np.int32)
    x2 = np.zeros((n_new,) + x.shape[1:]); v2 = np.zeros((n_new,) + v.shape[1:])
    f2 = np.zeros(n_new, np.int32); E2 = np.zeros(n_new)
    _orc._load().orc_gather(t.ref, len(counts), _orc._p(counts), _orc._p(x), _orc._p(v),
                            _orc._p(fam), _orc._p(E), vscale, _orc._p(x2), _orc._p(v2),
                            _orc._p(f2), _orc._p(E2))
    return x2, v2, f2, E2


def observables(top, x, v, fam, E, n_init):
    """The C oracle's observables of a population of any size; families are
    counted among the n_init slots of the start population."""
    o = _orc.observables(top, x, v, fam, E)
    o["n_families"] = int(len(np.unique(fam[(fam >= 0) & (fam < n_init)])))
    o["R"] = int(len(E))
    return o


def anneal(top, R_target, temps, theta, dt, gamma, seed, rule, mol=0, n_threads=None):
    """PAMD with a variable population: the PAMD scheme's steps in order with
    the nearest-integer (rule = 'nearest') or Poisson (rule = 'poisson') copy
    numbers.  Returns the list of per-temperature observable dicts (with the
    population size "R", ln Q and the running sum of ln Q)."""
    counts_of = {"nearest": nearest_integer_counts, "poisson": poisson_counts}[rule]
    x, v, fam = _orc.init(top, R_target, temps[0], seed, mol)
    step = 0
    x, v, E = _orc.propagate(top, x, v, theta, dt, temps[0], gamma, seed, step, mol, n_threads)
    step += theta
    o = observables(top, x, v, fam, E, R_target)
    o.update(T=float(temps[0]), lnQ=0.0, sum_lnQ=0.0)
    out = [o]
    s_lnq = 0.0
    for i in range(1, len(temps)):
        lnq, W = _orc.resample_weights(E, temps[i - 1], temps[i])
        cnt = counts_of(W, R_target, seed, i, mol)
        if cnt.sum() == 0:
            raise RuntimeError("the population died out")
        x, v, fam, E = gather(top, cnt, x, v, fam, E, math.sqrt(temps[i] / temps[i - 1]))
        x, v, E = _orc.propagate(top, x, v, theta, dt, temps[i], gamma, seed, step, mol, n_threads)
        step += theta
        s_lnq += lnq
        o = observables(top, x, v, fam, E, R_target)
        o.update(T=float(temps[i]), lnQ=float(lnq), sum_lnQ=s_lnq, max_copies=int(cnt.max()))
        out.append(o)
    return out
