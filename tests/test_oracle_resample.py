"""Pins of the oracle's resampling step (PAMD scheme, step 2, and the paragraph
on multinomial resampling) and of its observables.

* The target->ancestor map hits ancestor j exactly W_j times (brute force).
* E[n_j] = tau_j, with the multinomial variance (Monte Carlo z-test).
* sum_j n_j = R for every draw; zero copies prune.
* ln Q against the exact log-mean-exp from mpmath; special cases
  (T_next = T_prev gives ln Q = 0; constant energies give uniform weights).
* Integer weights against floor(2^s exp(a_j - max a)) computed exactly.
* Velocity rescaling by sqrt(T_i/T_{i-1}): with theta = 0 the measured
  temperature follows the schedule.
* The family-binned jackknife error equals the textbook standard error of
  the bin means when all bins have the same size.
"""
import math

import numpy as np
import pytest

import pamd_inputs as pi

KB = 0.008314462618


def test_ancestor_map_brute_force(orc):
    for W in ([3, 0, 5, 1, 2], [1], [0, 0, 7], [4, 4, 4, 4], [1, 0, 0, 0, 1]):
        W = np.array(W, np.uint64)
        C = np.cumsum(W)
        hits = np.zeros(len(W), int)
        for t in range(int(C[-1])):
            hits[orc.ancestor(C, t)] += 1
        np.testing.assert_array_equal(hits, W)


def test_weight_shift_keeps_sum_below_2_63(orc):
    for R, s in [(1, 63), (2, 62), (3, 61), (4, 61), (5, 60), (256, 55), (2**20, 43), (2**20 + 1, 42)]:
        assert orc.weight_shift(R) == s
        E = np.zeros(R) if R < 5000 else np.zeros(16)
        if R < 5000:
            _, W = orc.resample_weights(E, 300.0, 290.0)
            total = sum(int(w) for w in W)
            assert total <= 2**63 and all(int(w) == 2**s for w in W)


def test_counts_sum_to_R_and_prune(orc):
    E = pi.random_energies(200, -100.0, 30.0, 3)
    lnq, W = orc.resample_weights(E, 800.0, 700.0)
    for ti in range(1, 40):
        n = orc.multinomial_counts(W, 12345, ti)
        assert n.sum() == 200 and n.min() >= 0
    # very low weights are never copied
    E2 = np.array([0.0, 0.0, 1e5, 1e5])
    _, W2 = orc.resample_weights(E2, 800.0, 700.0)
    assert int(W2[2]) == 0 and int(W2[3]) == 0
    for ti in range(1, 50):
        n = orc.multinomial_counts(W2, 7, ti)
        assert n[2] == 0 and n[3] == 0


def test_expected_copies_equal_tau(orc):
    R = 6
    E = np.array([-30.0, -10.0, 0.0, 5.0, 12.0, 40.0])
    Tp, Tn = 500.0, 400.0
    dbeta = 1 / (KB * Tn) - 1 / (KB * Tp)
    w = np.exp(-dbeta * (E - E.min()))
    tau = R * w / w.sum()
    lnq, W = orc.resample_weights(E, Tp, Tn)
    M = 20000
    counts = np.array([orc.multinomial_counts(W, 99, ti) for ti in range(1, M + 1)])
    mean = counts.mean(0)
    p = tau / R
    se = np.sqrt(R * p * (1 - p) / M)
    z = (mean - tau) / se
    assert np.abs(z).max() < 4.5, z
    var = counts.var(0)
    assert np.all(np.abs(var / (R * p * (1 - p)) - 1) < 0.06)


def test_lnq_against_exact_log_mean_exp(orc):
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 200
    for seed, R, Tp, Tn in [(1, 50, 1000.0, 950.0), (2, 1000, 400.0, 300.0), (3, 7, 300.0, 310.0)]:
        E = pi.random_energies(R, 250.0, 40.0, seed)
        lnq, W = orc.resample_weights(E, Tp, Tn)
        dbeta = mp.mpf(1) / (mp.mpf(KB) * Tn) - mp.mpf(1) / (mp.mpf(KB) * Tp)
        exact = mp.log(mp.fsum(mp.exp(-dbeta * mp.mpf(float(e))) for e in E) / R)
        assert abs(lnq - float(exact)) < 1e-11 * max(1.0, abs(float(exact)))
        # integer weights: floor(2^s e^(a_j - max a)) up to the rounding of the
        # double-precision reduction a_j - max a (relative 2^-50)
        s = orc.weight_shift(R)
        dbf = 1 / (KB * Tn) - 1 / (KB * Tp)
        a = -dbf * E
        m = a.max()
        for j in range(R):
            ex = mp.floor(mp.mpf(2) ** s * mp.exp(mp.mpf(float(a[j] - m))))
            assert abs(int(W[j]) - int(ex)) <= max(2.0, float(ex) * 2.0**-50)


def test_lnq_special_cases(orc):
    E = pi.random_energies(33, 10.0, 5.0, 1)
    lnq, W = orc.resample_weights(E, 345.0, 345.0)
    assert lnq == 0.0
    assert len(set(int(w) for w in W)) == 1
    Ec = np.full(40, -12.5)
    lnq, W = orc.resample_weights(Ec, 500.0, 450.0)
    dbeta = 1 / (KB * 450.0) - 1 / (KB * 500.0)
    assert lnq == -dbeta * -12.5
    assert len(set(int(w) for w in W)) == 1


def test_resample_uniforms_are_uniform(orc):
    u = np.array([orc.resample_uniform(5, k, 3) for k in range(20000)], dtype=np.float64) / 2.0**64
    assert abs(u.mean() - 0.5) < 4 * math.sqrt(1 / 12 / len(u))
    hist = np.histogram(u, bins=20, range=(0, 1))[0]
    chi2 = ((hist - len(u) / 20) ** 2 / (len(u) / 20)).sum()
    assert chi2 < 50  # 19 degrees of freedom
    assert orc.resample_uniform(5, 0, 3) != orc.resample_uniform(5, 0, 4)


def test_gather_order_recentre_and_scale(orc):
    top = pi.make_chain(5, 1)
    R = 4
    x = pi.perturbed_positions(top, R, 0.05, 1) + np.arange(R)[:, None, None]
    v = pi.gaussian_velocities(R, 5, 1.0, 2)
    fam = np.array([10, 11, 12, 13], np.int32)
    E = np.array([1.0, 2.0, 3.0, 4.0])
    counts = np.array([0, 3, 0, 1], np.int32)
    x2, v2, f2, E2 = orc.gather(top, counts, x, v, fam, E, 0.5)
    np.testing.assert_array_equal(f2, [11, 11, 11, 13])
    np.testing.assert_array_equal(E2, [2.0, 2.0, 2.0, 4.0])
    np.testing.assert_allclose(v2[0], 0.5 * v[1])
    np.testing.assert_allclose(v2[3], 0.5 * v[3])
    com = (x2 * top.mass[None, :, None]).sum(1) / top.mass.sum()
    assert np.abs(com).max() < 1e-12
    np.testing.assert_allclose(x2[1] - x2[1].mean(0), x[1] - x[1].mean(0), atol=1e-12)


def test_velocity_rescaling_follows_schedule(orc):
    top = pi.make_chain(6, 3)
    temps = pi.geometric_schedule(900.0, 300.0, 5)
    obs, *_ = orc.anneal(top, 4000, temps, 0, 0.001, 1.0, 3)
    tm = np.array([o["t_meas"] for o in obs])
    se = tm * math.sqrt(2.0 / (3 * 6 * 4000))
    assert np.all(np.abs(tm - temps) < 5 * se), (tm, temps)


def test_observables_binning_and_closed_forms(orc):
    top = pi.make_chain(7, 2)
    R = 64 * 10
    rng = np.random.default_rng(4)
    E = rng.normal(3.0, 2.0, R)
    fam = np.arange(R, dtype=np.int32)
    # straight line, spacing a: R_g^2 = a^2 (N^2 - 1) / 12
    a = 0.2
    line = np.zeros((7, 3)); line[:, 2] = a * np.arange(7)
    x = np.repeat(line[None], R, 0)
    v = np.zeros((R, 7, 3)); v[:, 0, 0] = 2.0
    o = orc.observables(top, x, v, fam, E)
    assert abs(o["rg2"] - a * a * 48 / 12) < 1e-12 and o["rg_se"] < 1e-12
    assert abs(o["e_kin"] - 0.5 * 12.0 * 4.0) < 1e-12
    assert abs(o["t_meas"] - 2 * o["e_kin"] / (3 * 7 * KB)) < 1e-9
    bins = np.array([E[fam % 64 == b].mean() for b in range(64)])
    assert abs(o["e_pot"] - E.mean()) < 1e-12
    assert abs(o["e_pot_se"] - bins.std(ddof=1) / 8.0) < 1e-12
    assert o["n_families"] == R
    # one family only: no error estimate is possible
    o1 = orc.observables(top, x, v, np.zeros(R, np.int32), E)
    assert o1["e_pot_se"] == 0.0 and o1["n_families"] == 1
