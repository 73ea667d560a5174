"""Pins of the adaptive-temperature and systematic-resampling oracle
(oracle/adaptive.py): the overlap of two canonical Gamma energy distributions
in closed form, special cases, the floor/ceil property of systematic counts,
and the geometric schedule the overlap condition must produce for a harmonic
chain."""
import math

import numpy as np
import pytest

import oracle as orc
import pamd_inputs as pi
from oracle import adaptive as A

KB = A.KB


def _gamma_overlap(k, T1, T2):
    """Exact overlap sum_E min(P_T1, P_T2) of Gamma(k, k_B T) energy densities, T2 < T1."""
    from scipy.special import gammainc
    b1, b2 = 1.0 / (KB * T1), 1.0 / (KB * T2)
    Es = k * math.log(b2 / b1) / (b2 - b1)  # the densities cross once, at Es
    return gammainc(k, b1 * Es) + 1.0 - gammainc(k, b2 * Es)


def test_overlap_special_cases():
    rng = np.random.default_rng(0)
    E = rng.normal(-100.0, 5.0, 1000)
    assert A.overlap(E, 0.0) == 1.0
    assert A.overlap(np.full(50, 3.0), 7.5) == 1.0
    grid = np.linspace(0.0, 2.0, 41)
    a = [A.overlap(E, d) for d in grid]
    assert all(x >= y for x, y in zip(a, a[1:]))
    assert a[-1] < 0.05


@pytest.mark.parametrize("k,T1,T2", [(7.5, 400.0, 360.0), (7.5, 400.0, 300.0), (30.0, 1000.0, 900.0)])
def test_overlap_estimates_the_gamma_closed_form(k, T1, T2):
    rng = np.random.default_rng(int(k * 10 + T2))
    E = rng.gamma(k, KB * T1, 400000)
    d = 1.0 / (KB * T2) - 1.0 / (KB * T1)
    assert abs(A.overlap(E, d) - _gamma_overlap(k, T1, T2)) < 0.005


def test_next_temperature_meets_the_target_or_stops_at_the_end():
    rng = np.random.default_rng(3)
    E = rng.gamma(20.0, KB * 800.0, 20000)
    T, a = A.next_temperature(E, 800.0, 300.0, 0.6)
    assert 300.0 < T < 800.0 and abs(a - 0.6) < 1e-12
    T2, a2 = A.next_temperature(E, 800.0, 780.0, 0.6)
    assert T2 == 780.0 and a2 >= 0.6


def test_systematic_counts_are_floor_or_ceil_of_the_expected_copies():
    rng = np.random.default_rng(5)
    for R in (1, 7, 64, 1000):
        E = rng.normal(0.0, 20.0, R)
        _, W = orc.resample_weights(E, 500.0, 400.0)
        for ti in range(1, 4):
            n = A.systematic_counts(W, 99, ti)
            assert n.sum() == R
            exp = R * np.array([int(w) for w in W], dtype=np.float64) / float(sum(int(w) for w in W))
            assert np.all((n == np.floor(exp)) | (n == np.ceil(exp))), (R, ti)


def test_systematic_counts_equal_weights_and_mean():
    n = A.systematic_counts(np.full(16, 1 << 40, np.uint64), 1, 1)
    np.testing.assert_array_equal(n, np.ones(16, np.int32))
    # E[n_j] = R W_j / C over the uniform: average over resampling indices
    W = np.array([1, 2, 3, 10, 0, 4], np.uint64) << np.uint64(50)
    m = np.mean([A.systematic_counts(W, 7, i) for i in range(1, 3001)], axis=0)
    expect = 6 * W.astype(np.float64) / float(W.astype(np.float64).sum())
    assert np.all(np.abs(m - expect) < 0.03), m - expect


def test_adaptive_anneal_of_a_harmonic_chain_is_geometric():
    """For Gamma(k) energy distributions the overlap depends on T2/T1 only, so
    the overlap condition picks a constant ratio: the schedule is geometric
    with the ratio solving the closed-form overlap = alpha*."""
    from scipy.optimize import brentq
    n, kb = 6, 400.0
    k = 1.5 * (n - 1)
    top = pi.make_harmonic_chain(n, kb, 0.0)
    alpha = 0.5
    obs, temps, energies = A.anneal_adaptive(top, 2048, 400.0, 150.0, alpha, 100, 0.002, 5.0, 21, 40)
    r_exact = brentq(lambda r: _gamma_overlap(k, 1.0, r) - alpha, 1e-6, 1.0 - 1e-9)
    ratios = temps[1:] / temps[:-1]
    assert temps[-1] == 150.0 and np.all(np.diff(temps) < 0)
    assert np.all(np.abs(ratios[:-1] - r_exact) < 0.03), (ratios, r_exact)
    e = np.array([o["e_pot"] for o in obs]); se = np.array([o["e_pot_se"] for o in obs])
    assert np.all(np.abs(e - k * KB * temps) < 4 * se + 0.01 * k * KB * temps)
