"""FP64 CPU oracle of the multiple-histogram reweighting (WHAM) refinement --
TEST INFRASTRUCTURE.

Only the test suite and the benchmark's CPU legs use this module.  Plain numpy
in float64, written from the definitions below; it shares no code with the
CUDA library.

Free-energy paragraph of the paper: the running sum of ln Q estimates
ln Z(T_i) - ln Z(T_0) of the configurational partition function, and those
values start a few sweeps of the self-consistency equations of the
multiple-histogram method (Ferrenberg & Swendsen 1989; Kumar et al. 1992).
For canonical samples at inverse temperatures beta_i = 1 / (k_B T_i),
i = 0..K, N_i samples at beta_i, energy histograms H_i(b) on common bins with
centres E_b and H(b) = sum_i H_i(b):

  g_b   = H(b) / sum_i N_i exp(-beta_i E_b - ln Z_i)     (density of states of bin b)
  Z_i   = sum_b g_b exp(-beta_i E_b)

One sweep evaluates the first line from the current ln Z_i and then the
second; afterwards the gauge ln Z_0 = 0 is restored by subtracting the new
ln Z_0 from every ln Z_i.  The sweeps stop after max_iter, or once the largest
change of an ln Z_i in a sweep is below tol.  Every sum of exponentials is
taken as max + ln(sum exp(x - max)).

Binning (a reading: the paper does not state one): n_bins equal bins over
[e_min, e_max], w = (e_max - e_min) / n_bins, centres E_b = e_min + (b + 1/2) w;
a sample E goes to bin floor((E - e_min) * (n_bins / (e_max - e_min))), the
top edge to the last bin; samples outside [e_min, e_max] or not finite are
not counted, and N_i counts the samples that were.  When the range comes from
the data it is [min E, max E] over the finite samples, widened to
[min E, min E + 1] if all of them are equal.

Reweighting to any temperature T from the final g_b:
  ln Z(T) = ln sum_b g_b exp(-E_b / k_B T),
  <E>(T)  = sum_b E_b p_b,   var E(T) = sum_b (E_b - <E>)^2 p_b,
  p_b     = g_b exp(-E_b / k_B T) / Z(T).
"""
from __future__ import annotations

import numpy as np

KB = 0.008314462618


def _lse(x):
    """ln sum exp(x) over the last axis; -inf where every entry is -inf."""
    x = np.asarray(x, dtype=np.float64)
    m = np.max(x, axis=-1, keepdims=True)
    safe = np.where(np.isfinite(m), m, 0.0)
    s = np.sum(np.exp(x - safe), axis=-1, keepdims=True)
    with np.errstate(divide="ignore"):
        out = np.log(s) + safe
    return np.where(np.isfinite(m), out, -np.inf)[..., 0]


def energy_range(E):
    """[min, max] of the finite energies, widened to a unit range if they are equal."""
    E = np.asarray(E, dtype=np.float64)
    f = E[np.isfinite(E)]
    lo, hi = float(f.min()), float(f.max())
    if not hi > lo:
        hi = lo + 1.0
    return lo, hi


def histograms(E, n_bins, e_min, e_max):
    """Counts H[i, b] of the energies E[i, :] (one row per temperature)."""
    E = np.asarray(E, dtype=np.float64)
    inv = n_bins / (e_max - e_min)
    H = np.zeros((E.shape[0], n_bins), dtype=np.int64)
    for i in range(E.shape[0]):
        e = E[i][np.isfinite(E[i])]
        e = e[(e >= e_min) & (e <= e_max)]
        b = np.floor((e - e_min) * inv).astype(np.int64)
        b = np.minimum(b, n_bins - 1)
        H[i] = np.bincount(b, minlength=n_bins)
    return H


def bin_centres(n_bins, e_min, e_max):
    w = (e_max - e_min) / n_bins
    return e_min + (np.arange(n_bins) + 0.5) * w


def ln_dos(H, beta, Eb, lnZ):
    """ln g_b from the histograms and the current ln Z_i (-inf for empty bins)."""
    H = np.asarray(H, dtype=np.float64)
    Htot = H.sum(axis=0)
    N = H.sum(axis=1)
    lnN = np.full(N.shape, -np.inf)
    lnN[N > 0] = np.log(N[N > 0])
    # den_b = ln sum_i N_i exp(-beta_i E_b - ln Z_i)
    terms = lnN[None, :] - np.outer(Eb, beta) - np.asarray(lnZ)[None, :]
    den = _lse(terms)
    with np.errstate(divide="ignore"):
        lnH = np.log(Htot)
    return np.where(Htot > 0, lnH - den, -np.inf)


def ln_partition(ln_g, beta, Eb):
    """ln Z_i = ln sum_b g_b exp(-beta_i E_b)."""
    return _lse(np.asarray(ln_g)[None, :] - np.outer(beta, Eb))


def iterate(H, T, Eb, lnZ_init=None, max_iter=100, tol=1e-10):
    """Self-consistency sweeps.  Returns (ln Z [K+1], ln g [n_bins], sweeps, last change)."""
    beta = 1.0 / (KB * np.asarray(T, dtype=np.float64))
    lnZ = np.zeros(len(beta)) if lnZ_init is None else np.array(lnZ_init, dtype=np.float64)
    lnZ = lnZ - lnZ[0]
    sweeps, delta = 0, np.inf
    for _ in range(max_iter):
        ln_g = ln_dos(H, beta, Eb, lnZ)
        new = ln_partition(ln_g, beta, Eb)
        new = new - new[0]
        delta = float(np.max(np.abs(new - lnZ)))
        lnZ = new
        sweeps += 1
        if delta < tol:
            break
    return lnZ, ln_dos(H, beta, Eb, lnZ), sweeps, delta


def reweight(ln_g, Eb, T_eval):
    """(ln Z(T), <E>(T), var E(T)) at each temperature of T_eval."""
    ln_g = np.asarray(ln_g, dtype=np.float64)
    out = []
    for T in np.atleast_1d(T_eval):
        beta = 1.0 / (KB * T)
        x = ln_g - beta * Eb
        lz = float(_lse(x))
        p = np.exp(x - lz)
        m = float(np.sum(Eb * p))
        v = float(np.sum((Eb - m) ** 2 * p))
        out.append((lz, m, v))
    a = np.array(out)
    return a[:, 0], a[:, 1], a[:, 2]


def wham(E, T, n_bins, e_min=None, e_max=None, lnZ_init=None, max_iter=100, tol=1e-10, T_eval=None):
    """Histograms of E[i, :] sampled at T[i], then the sweeps; a dict of the results."""
    if e_min is None or e_max is None or not e_max > e_min:
        e_min, e_max = energy_range(E)
    H = histograms(E, n_bins, e_min, e_max)
    Eb = bin_centres(n_bins, e_min, e_max)
    lnZ, ln_g, sweeps, delta = iterate(H, T, Eb, lnZ_init, max_iter, tol)
    out = {"hist": H, "e_min": e_min, "bin_width": (e_max - e_min) / n_bins, "lnZ": lnZ,
           "ln_g": ln_g, "iterations": sweeps, "max_delta": delta}
    if T_eval is not None:
        out["lnZ_eval"], out["e_mean_eval"], out["e_var_eval"] = reweight(ln_g, Eb, T_eval)
    return out
