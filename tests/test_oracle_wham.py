"""Pins of the WHAM oracle (oracle/wham.py) against results fixed by the
mathematics: exact histograms of a known density of states, the harmonic
chain's closed-form free energies, special cases and binning invariants."""
import math

import numpy as np

from oracle import wham as W

KB = W.KB


def _exact_hist(ln_g, Eb, T, N):
    """Expected (real-valued) counts N_i g_b exp(-beta_i E_b) / Z_i and the true ln Z_i."""
    beta = 1.0 / (KB * np.asarray(T))
    lnZ = np.array([math.log(sum(math.exp(lg - b * e) for lg, e in zip(ln_g, Eb))) for b in beta])
    H = np.array([[n * math.exp(lg - b * e - lz) for lg, e in zip(ln_g, Eb)]
                  for n, b, lz in zip(N, beta, lnZ)])
    return H, lnZ


def test_exact_histograms_give_the_true_partition_functions():
    # density of states of a 6-dimensional harmonic system, E^(d/2 - 1), on 300 bins
    Eb = W.bin_centres(300, 0.0, 60.0)
    ln_g = 2.0 * np.log(Eb)
    T = np.array([600.0, 450.0, 350.0, 280.0, 220.0])
    N = np.array([1000.0, 2000.0, 1500.0, 3000.0, 800.0])
    H, lnZ_true = _exact_hist(ln_g, Eb, T, N)
    lnZ, lg, sweeps, delta = W.iterate(H, T, Eb, None, max_iter=5000, tol=1e-13)
    assert delta < 1e-13 and sweeps < 5000
    np.testing.assert_allclose(lnZ, lnZ_true - lnZ_true[0], atol=1e-9)
    # the density of states up to one additive constant
    d = lg - ln_g
    np.testing.assert_allclose(d - d[0], 0.0, atol=1e-9)


def test_the_true_partition_functions_are_a_fixed_point():
    Eb = W.bin_centres(50, -40.0, 10.0)
    ln_g = 0.05 * (Eb + 40.0) ** 1.5
    T = np.array([900.0, 700.0, 500.0])
    N = np.array([500.0, 500.0, 500.0])
    H, lnZ_true = _exact_hist(ln_g, Eb, T, N)
    lnZ, _, sweeps, delta = W.iterate(H, T, Eb, lnZ_true, max_iter=1, tol=0.0)
    assert sweeps == 1 and delta < 1e-11
    np.testing.assert_allclose(lnZ, lnZ_true - lnZ_true[0], atol=1e-11)


def test_harmonic_chain_closed_form():
    """Bond-only chain with r0 = 0: E ~ Gamma(d/2, k_B T), d = 3(N - 1);
    ln Z(T_i) - ln Z(T_0) = (d/2) ln(T_i / T_0) and <E>(T) = (d/2) k_B T."""
    n_atoms = 6
    d = 3 * (n_atoms - 1)
    T = np.geomspace(400.0, 200.0, 7)
    rng = np.random.default_rng(5)
    E = np.stack([rng.gamma(d / 2, KB * t, 40000) for t in T])
    out = W.wham(E, T, 400, max_iter=2000, tol=1e-12, T_eval=[300.0, 250.0])
    exact = 0.5 * d * np.log(T / T[0])
    assert np.max(np.abs(out["lnZ"] - exact)) < 0.03, out["lnZ"] - exact
    np.testing.assert_allclose(out["e_mean_eval"], 0.5 * d * KB * np.array([300.0, 250.0]), rtol=0.01)
    # variance of a Gamma(d/2, k_B T) energy: (d/2) (k_B T)^2
    np.testing.assert_allclose(out["e_var_eval"], 0.5 * d * (KB * np.array([300.0, 250.0])) ** 2, rtol=0.05)


def test_single_temperature_reweights_to_the_histogram_mean():
    rng = np.random.default_rng(1)
    E = rng.normal(-50.0, 3.0, (1, 5000))
    out = W.wham(E, [310.0], 64, max_iter=3, tol=0.0, T_eval=[310.0])
    Eb = W.bin_centres(64, out["e_min"], out["e_min"] + 64 * out["bin_width"])
    H = out["hist"][0]
    assert out["lnZ"][0] == 0.0
    assert abs(out["e_mean_eval"][0] - float(np.sum(Eb * H) / H.sum())) < 1e-10


def test_binning_invariants():
    e_min, e_max, nb = -3.0, 5.0, 16
    w = (e_max - e_min) / nb
    want = np.arange(nb) % 5
    centres = W.bin_centres(nb, e_min, e_max)
    samples = np.repeat(centres, want)
    extra = np.array([e_min, e_max, e_max + 1e-9, e_min - 1.0, np.nan, np.inf])
    E = np.concatenate([samples, extra])[None, :]
    H = W.histograms(E, nb, e_min, e_max)[0]
    expect = want.copy()
    expect[0] += 1        # the bottom edge
    expect[-1] += 1       # the top edge goes to the last bin
    np.testing.assert_array_equal(H, expect)
    assert abs(centres[1] - centres[0] - w) < 1e-15


def test_degenerate_range_is_widened():
    E = np.full((2, 10), 7.25)
    lo, hi = W.energy_range(E)
    assert (lo, hi) == (7.25, 8.25)
    H = W.histograms(E, 4, lo, hi)
    np.testing.assert_array_equal(H, [[10, 0, 0, 0], [10, 0, 0, 0]])
