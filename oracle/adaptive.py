"""FP64 CPU oracle of the adaptive temperature step and of systematic
resampling -- TEST INFRASTRUCTURE.

Only the test suite and the benchmark's CPU legs use this module.  Plain numpy
/ Python integers written from the definitions below; the anneal driver
composes the C oracle's own steps (oracle/__init__.py).  Nothing is shared
with the CUDA library.

Overlap condition (temperature-choice sentence of the PAMD scheme: the
temperatures follow the rules of parallel tempering, i.e. enough overlap of
the energy histograms, and can be chosen automatically from an overlap
condition).  For a population with potential energies E_j, j < R, at
beta = 1/(k_B T_prev) and a lower temperature T with dbeta = 1/(k_B T) - beta:
    tau_j(dbeta) = R exp(-dbeta E_j) / sum_k exp(-dbeta E_k)
    alpha(dbeta) = (1/R) sum_j min(1, tau_j(dbeta)),
the population estimate of the overlap sum_E min(P_T_prev(E), P_T(E)) of the
two canonical energy distributions (Barash et al. 2017).  alpha(0) = 1 and it
falls as dbeta grows.  The next temperature is T_final when
alpha(dbeta_final) >= alpha*, and otherwise the T whose alpha equals alpha*
(a root found by Brent's method, scipy.optimize.brentq, to 1e-15 relative).

Systematic resampling (one of the resampling implementations the paper cites
besides the multinomial draws it uses): with the integer weights W_j and
inclusive sums C_j of the multinomial realisation, C = C_{R-1}, one 64-bit
uniform U (the multinomial's draw for slot 0) and V = floor(U C / 2^64), new
slot k takes target t_k = floor((k C + V) / R) and ancestor = the first j with
C_j > t_k.  Each n_j is then floor(R W_j / C) or that plus one.
"""
from __future__ import annotations

import numpy as np

import oracle as _orc

KB = 0.008314462618


def overlap(E, dbeta):
    """alpha(dbeta) of the energies E (FP64)."""
    E = np.asarray(E, dtype=np.float64)
    R = len(E)
    a = -dbeta * (E - E.min())
    w = np.exp(a)
    tau = R * w / w.sum()
    return float(np.minimum(1.0, tau).mean())


def next_temperature(E, T_prev, T_final, alpha_target):
    """(T_next, alpha(T_next)) from the overlap condition."""
    from scipy.optimize import brentq
    beta = 1.0 / (KB * T_prev)
    d_final = 1.0 / (KB * T_final) - beta
    a_final = overlap(E, d_final)
    if a_final >= alpha_target:
        return float(T_final), a_final
    d = brentq(lambda x: overlap(E, x) - alpha_target, 0.0, d_final, xtol=1e-15 * d_final,
               rtol=1e-15, maxiter=500)
    return float(1.0 / (KB * (beta + d))), overlap(E, d)


def systematic_counts(W, seed, temp_index, mol=0):
    """Copy counts n_j of systematic resampling with integer weights W (u64)."""
    W = [int(w) for w in np.asarray(W, dtype=np.uint64)]
    R = len(W)
    C = np.cumsum(np.asarray(W, dtype=object))
    total = int(C[-1])
    U = int(_orc.resample_uniform(seed, 0, temp_index, mol))
    V = (U * total) >> 64
    cnt = np.zeros(R, np.int32)
    j = 0
    for k in range(R):  # targets increase with k, so the ancestor index only moves forward
        t = (k * total + V) // R
        while int(C[j]) <= t:
            j += 1
        cnt[j] += 1
    return cnt


def anneal_adaptive(top, R, T0, T_final, alpha_target, theta, dt, gamma, seed, max_steps, mol=0,
                    n_threads=None):
    """PAMD run whose temperatures come from the overlap condition.  Returns
    (list of observable dicts, temperatures, energies at each temperature)."""
    x, v, fam = _orc.init(top, R, T0, seed, mol)
    step = 0
    x, v, E = _orc.propagate(top, x, v, theta, dt, T0, gamma, seed, step, mol, n_threads)
    step += theta
    obs = [_orc.observables(top, x, v, fam, E)]
    temps, energies = [float(T0)], [E.copy()]
    T = float(T0)
    for i in range(1, max_steps + 1):
        if T <= T_final:
            break
        Tn, _ = next_temperature(E, T, T_final, alpha_target)
        lnq, W = _orc.resample_weights(E, T, Tn)
        cnt = _orc.multinomial_counts(W, seed, i, mol)
        x, v, fam, E = _orc.gather(top, cnt, x, v, fam, E, np.sqrt(Tn / T))
        x, v, E = _orc.propagate(top, x, v, theta, dt, Tn, gamma, seed, step, mol, n_threads)
        step += theta
        T = Tn
        obs.append(_orc.observables(top, x, v, fam, E))
        temps.append(T)
        energies.append(E.copy())
    return obs, np.array(temps), energies
