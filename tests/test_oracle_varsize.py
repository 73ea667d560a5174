"""Pins of the variable-population resampling oracle (oracle/varsize.py).

* nearest integer: every n_j is floor(tau_j) or ceil(tau_j) of the exact
  rational tau_j = R_t W_j / C; equal weights give exactly R_t / R~ copies;
  over many resampling indices the mean of n_j is tau_j and the variance of
  the total is sum_j f_j (1 - f_j), f_j = frac(tau_j) (Bernoulli rounding);
* Poisson: the inversion sampler returns the quantile of SciPy's Poisson
  CDF; over many resampling indices n_j has mean and variance tau_j and the
  total has mean and variance R_t; chunked means (lambda > 500) keep them;
* a whole anneal of a harmonic chain with either rule gives the closed-form
  <E_pot>(T) = (3/2)(N-1) k_B T and sum ln Q = (3/2)(N-1) ln(T/T0).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import pamd_inputs as pi
from oracle import varsize as ov

KB = 0.008314462618


def _weights(orc, R, spread, seed, Tp=600.0, Tn=560.0):
    E = pi.random_energies(R, -30.0, spread, seed)
    return orc.resample_weights(E, Tp, Tn)[1]


def test_nearest_integer_is_floor_or_ceil(orc):
    W = _weights(orc, 300, 8.0, 1)
    C = sum(int(w) for w in W)
    for R_t in (300, 257, 1000):
        cnt = ov.nearest_integer_counts(W, R_t, 5, 3)
        for w, n in zip(W, cnt):
            tau = Fraction(R_t * int(w), C)
            assert math.floor(tau) <= n <= math.ceil(tau)


def test_nearest_integer_equal_weights_is_exact(orc):
    W = np.full(128, 1 << 50, dtype=np.uint64)
    assert np.all(ov.nearest_integer_counts(W, 128, 9, 1) == 1)
    assert np.all(ov.nearest_integer_counts(W, 384, 9, 1) == 3)
    assert ov.nearest_integer_counts(W, 128, 9, 1).sum() == 128


def test_nearest_integer_mean_and_total_variance(orc):
    W = _weights(orc, 40, 3.0, 2)
    R_t = 40
    C = sum(int(w) for w in W)
    tau = np.array([R_t * int(w) / C for w in W])
    f = tau - np.floor(tau)
    runs = np.array([ov.nearest_integer_counts(W, R_t, 77, i) for i in range(1, 4001)])
    z = (runs.mean(0) - tau) / np.sqrt(f * (1 - f) / len(runs) + 1e-300)
    assert np.all(np.abs(z[f > 0]) < 4.5)
    var_tot = (f * (1 - f)).sum()
    assert abs(runs.sum(1).var() / var_tot - 1.0) < 0.15


@pytest.mark.parametrize("lam", [0.05, 0.7, 3.0, 42.0, 480.0])
def test_poisson_inverse_is_the_scipy_quantile(lam):
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(int(lam * 100))
    for u in rng.uniform(0.0, 1.0, 400):
        n = ov.poisson_inverse(lam, float(u))
        lo = stats.poisson.cdf(n - 1, lam) if n > 0 else 0.0
        hi = stats.poisson.cdf(n, lam)
        # F(n-1) < u <= F(n), up to the FP64 rounding of the running sum
        assert lo - 1e-12 < u <= hi + 1e-12, (lam, u, n, lo, hi)


def test_poisson_counts_moments(orc):
    W = _weights(orc, 30, 2.0, 4)
    R_t = 30
    C = sum(int(w) for w in W)
    tau = np.array([(float(R_t) * float(int(w))) / float(C) for w in W])
    runs = np.array([ov.poisson_counts(W, R_t, 123, i) for i in range(1, 3001)])
    z = (runs.mean(0) - tau) / np.sqrt(tau / len(runs))
    assert np.all(np.abs(z) < 4.5)
    v = runs.var(0, ddof=1)
    assert np.all(np.abs(v / tau - 1.0) < 0.25)
    tot = runs.sum(1)
    assert abs(tot.mean() - R_t) < 4.5 * math.sqrt(R_t / len(runs))
    assert abs(tot.var(ddof=1) / R_t - 1.0) < 0.12


def test_poisson_chunked_mean(orc):
    """One replica carries almost all the weight: lambda ~ R_t is drawn in
    chunks of at most 500, and the result still has mean and variance R_t."""
    R_t = 1500
    W = np.array([1 << 40] + [1] * 9, dtype=np.uint64)
    draws = np.array([ov.poisson_counts(W, R_t, 9, i)[0] for i in range(1, 1501)])
    lam = (float(R_t) * float(1 << 40)) / float((1 << 40) + 9)
    assert abs(draws.mean() - lam) < 4.5 * math.sqrt(lam / len(draws))
    assert abs(draws.var(ddof=1) / lam - 1.0) < 0.12


@pytest.mark.parametrize("rule", ["nearest", "poisson"])
def test_variable_population_anneal_harmonic_closed_forms(orc, rule):
    n, kb = 5, 300.0
    top = pi.make_harmonic_chain(n, kb, 0.0)
    temps = pi.geometric_schedule(500.0, 300.0, 4)
    # theta = 1500 steps of 2 fs is 15 friction times: every block relaxes
    runs = [ov.anneal(top, 400, temps, 1500, 0.002, 5.0, 21 + 11 * k, rule) for k in range(6)]
    e = np.array([[o["e_pot"] for o in r] for r in runs])
    se = np.array([[o["e_pot_se"] for o in r] for r in runs])
    e_mean = e.mean(0)
    e_se = np.maximum(e.std(0, ddof=1) / np.sqrt(len(runs)), np.sqrt((se ** 2).sum(0)) / len(runs))
    e_exact = 1.5 * (n - 1) * KB * temps
    assert np.all(np.abs(e_mean - e_exact) <= 3 * e_se), (e_mean - e_exact) / e_se
    f = np.array([[o["sum_lnQ"] for o in r] for r in runs]).mean(0)
    assert np.all(np.abs(f - 1.5 * (n - 1) * np.log(temps / temps[0])) < 0.1)
    sizes = np.array([[o["R"] for o in r] for r in runs])
    assert np.all(np.abs(sizes - 400) < 8 * math.sqrt(400) + 8)
