"""Pins of the oracle's integrator, initialisation and whole-anneal driver.

* gamma = 0 reduces BAOAB to velocity Verlet: the total energy is conserved
  and its fluctuation shrinks as dt^2.
* A free particle under the O step relaxes as an Ornstein-Uhlenbeck process:
  <v^2> after n steps = c1^(2n) v0^2 + (1 - c1^(2n)) kT/m exactly.
* Equipartition: <E_kin> = (3N/2) k_B T.
* Bonds-only harmonic chain (r0 = 0): <E_pot>(T) = (3/2)(N-1) k_B T and the
  free-energy estimate sum ln Q_i = (3/2)(N-1) ln(T_i/T_0) (configurational
  partition-function ratio of N-1 independent 3-D Gaussians).
"""
import math

import numpy as np
import pytest

import pamd_inputs as pi

KB = 0.008314462618


def _total_energy(orc, top, x, v):
    return orc.energy_forces(top, x)[0] + orc.kinetic(top, v)


def _nve_fluct(orc, top, dt, t_total):
    x = top.x0[None].copy()
    v = pi.gaussian_velocities(1, top.n_atoms, math.sqrt(KB * 300 / 12.0), 3)
    h0 = _total_energy(orc, top, x[0], v[0])
    hs = []
    n_chunks = 20
    steps = int(round(t_total / dt / n_chunks))
    for c in range(n_chunks):
        x, v, _ = orc.propagate(top, x, v, steps, dt, 300.0, 0.0, 1, c * steps, n_threads=1)
        hs.append(_total_energy(orc, top, x[0], v[0]))
    return np.max(np.abs(np.array(hs) - h0)), orc.kinetic(top, v[0])


def test_nve_energy_conservation_and_dt2_scaling(orc):
    top = pi.make_chain(12, 4)
    d1, ek = _nve_fluct(orc, top, 0.001, 2.0)
    d2, _ = _nve_fluct(orc, top, 0.0005, 2.0)
    assert d1 < 0.05 * max(ek, 1.0)
    ratio = d1 / d2
    assert 2.5 < ratio < 6.0, ratio


def test_ornstein_uhlenbeck_free_particle(orc):
    top = pi.make_chain(1, 0)
    R, n, dt, gamma, T = 20000, 5, 0.01, 5.0, 400.0
    x = np.zeros((R, 1, 3))
    v = np.full((R, 1, 3), 0.7)
    x, v, _ = orc.propagate(top, x, v, n, dt, T, gamma, 99, 0)
    c2n = math.exp(-2 * gamma * dt * n)
    kTm = KB * T / 12.0
    mean_v = math.exp(-gamma * dt * n) * 0.7
    var_exp = (1 - c2n) * kTm
    vv = v.reshape(-1)
    assert abs(vv.mean() - mean_v) < 5 * math.sqrt(var_exp / vv.size)
    assert abs(vv.var() - var_exp) < 5 * var_exp * math.sqrt(2.0 / vv.size)


def test_init_maxwell_boltzmann_and_recentred(orc):
    top = pi.make_chain(10, 3)
    x, v, fam = orc.init(top, 4000, 500.0, 7)
    np.testing.assert_array_equal(fam, np.arange(4000))
    com = (x * top.mass[None, :, None]).sum(1) / top.mass.sum()
    assert np.abs(com).max() < 1e-12
    np.testing.assert_allclose(x[5], x[0])
    var = v.var()
    assert abs(var - KB * 500 / 12.0) < 5 * KB * 500 / 12.0 * math.sqrt(2.0 / v.size)


def test_equipartition(orc):
    top = pi.make_chain(10, 6)
    R, T, dt, gamma = 512, 300.0, 0.001, 10.0
    x, v, fam = orc.init(top, R, T, 21)
    # the all-trans start collapses and heats the chain: burn in for 2 ps
    x, v, _ = orc.propagate(top, x, v, 2000, dt, T, gamma, 21, 0)
    ek = []
    for c in range(6):
        x, v, _ = orc.propagate(top, x, v, 300, dt, T, gamma, 21, 2000 + 300 * c)
        ek.append([orc.kinetic(top, v[k]) for k in range(R)])
    ek = np.array(ek)
    target = 1.5 * top.n_atoms * KB * T
    # BAOAB's kinetic energy carries an O(dt^2) bias below 1% at dt = 1 fs
    se = ek.mean(0).std() / math.sqrt(R)
    assert abs(ek.mean() - target) < 4 * se + 0.01 * target, (ek.mean(), target, se)


@pytest.mark.slow
def test_harmonic_chain_pa_closed_forms(orc):
    n, kb = 6, 400.0
    top = pi.make_harmonic_chain(n, kb, 0.0)
    temps = pi.geometric_schedule(400.0, 200.0, 6)
    runs = []
    for seed in (1, 2, 3, 4):
        obs, *_ = orc.anneal(top, 1500, temps, 200, 0.002, 5.0, seed)
        runs.append(obs)
    epot = np.array([[o["e_pot"] for o in r] for r in runs])
    slnq = np.array([[o["sum_lnQ"] for o in r] for r in runs])
    e_exact = 1.5 * (n - 1) * KB * temps
    f_exact = 1.5 * (n - 1) * np.log(temps / temps[0])
    e_se = epot.std(0, ddof=1) / 2.0 + 1e-12
    f_se = slnq.std(0, ddof=1) / 2.0 + 1e-12
    assert np.all(np.abs(epot.mean(0) - e_exact) < 4 * e_se + 0.01 * e_exact), (epot.mean(0), e_exact)
    assert np.all(np.abs(slnq.mean(0) - f_exact) < 4 * f_se + 0.01), (slnq.mean(0), f_exact)
    # the family-binned standard error is of the right size
    se_bin = np.array([[o["e_pot_se"] for o in r] for r in runs]).mean(0)
    assert np.all(se_bin[1:] < 5 * epot.std(0, ddof=1)[1:] + 1e-9)


def test_anneal_without_resampling_keeps_families(orc):
    top = pi.make_chain(8, 2)
    temps = pi.geometric_schedule(600.0, 400.0, 3)
    obs, x, v, fam, E = orc.anneal(top, 64, temps, 20, 0.001, 1.0, 5, resample=False)
    np.testing.assert_array_equal(fam, np.arange(64))
    assert all(o["n_families"] == 64 and o["max_copies"] == 1 for o in obs)
    obs2, *_ = orc.anneal(top, 64, temps, 20, 0.001, 1.0, 5, resample=True)
    assert obs2[-1]["n_families"] <= 64
    assert obs2[1]["lnQ"] == obs[1]["lnQ"]  # the first weights see the same population
