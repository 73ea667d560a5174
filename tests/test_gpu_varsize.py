"""Variable population size on the GPU (nearest-integer and Poisson
resampling) against the oracle (oracle/varsize.py).

* copy numbers bit-exact given the same energies and Philox stream, over two
  consecutive resamplings (the second from a population whose size is no
  longer the target), with ln Q to 1e-12 and the new live size equal to the
  sum of the copy numbers;
* the gathered population element-wise (positions recentred in FP32);
* Poisson means above the chunk size (one dominant replica) bit-exact;
* an empty population is reported as PAMD_EPOPSIZE;
* whole anneals of a harmonic chain: the closed-form <E_pot>(T) and
  sum ln Q within 3 standard errors over eight runs, every recorded
  population size equal to the live size, and the 22-atom chain against the
  oracle's anneal within 3 combined standard errors.
"""
import math

import numpy as np
import pytest

import pamd_inputs as pi
from oracle import varsize as ov

pytestmark = pytest.mark.gpu

KB = 0.008314462618
RULES = {"nearest": (2, ov.nearest_integer_counts), "poisson": (3, ov.poisson_counts)}


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_06016_gb300 import build, pamd
    build.build()
    pamd.load()
    return pamd


def _opts(lib, **kw):
    o = lib.pamd_options_default()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("rule", ["nearest", "poisson"])
@pytest.mark.parametrize("R,spread", [(1000, 20.0), (3000, 3.0), (37, 50.0)])
def test_varsize_counts_and_gather_match_oracle(lib, orc, rule, R, spread):
    code, counts_of = RULES[rule]
    n = 9
    top = pi.make_chain(n, 2)
    seed = 55 + R
    ctx = lib.pamd_init(top, R, 700.0, seed, _opts(lib, resample_rule=code))
    try:
        live, cap = lib.pamd_population_size(ctx)
        assert live == R and cap == R + 8 * math.ceil(math.sqrt(R)) + 64
        x = np.zeros((cap, n, 3)); v = np.zeros((cap, n, 3)); E = np.zeros(cap)
        x[:R] = f32(pi.perturbed_positions(top, R, 0.02, 5))
        v[:R] = f32(pi.gaussian_velocities(R, n, 0.5, 6))
        E[:R] = pi.random_energies(R, -50.0, spread, 8)
        fam = np.arange(cap, dtype=np.int32)
        lib.pamd_set_state(ctx, x, v, E, fam)
        temps = [700.0, 640.0, 600.0]
        R_cur, xo, vo, fo, Eo = R, x[:R], v[:R], fam[:R], E[:R]
        for i in (1, 2):
            cnt, lnq = lib.pamd_resample(ctx, temps[i - 1], temps[i])
            lnq_o, W = orc.resample_weights(Eo, temps[i - 1], temps[i])
            cnt_o = counts_of(W, R, seed, i)
            np.testing.assert_array_equal(cnt[:R_cur], cnt_o)
            assert abs(lnq - lnq_o) <= 1e-12 * max(1.0, abs(lnq_o))
            R_new = int(cnt_o.sum())
            assert lib.pamd_population_size(ctx)[0] == R_new
            xo, vo, fo, Eo = ov.gather(top, cnt_o, xo, vo, fo, Eo, math.sqrt(temps[i] / temps[i - 1]))
            xg, vg, eg, fg = lib.pamd_get_state(ctx)
            np.testing.assert_array_equal(fg[:R_new], fo)
            np.testing.assert_array_equal(eg[:R_new], Eo)
            assert np.abs(xg[:R_new] - xo).max() < 4e-6
            assert np.abs(vg[:R_new] - vo).max() <= 2e-7 * np.abs(vo).max()
            R_cur = R_new
    finally:
        lib.pamd_destroy(ctx)


def test_poisson_chunked_mean_matches_oracle(lib, orc):
    """One replica far below the others: its mean copy number exceeds the
    chunk size of 500 and is drawn in several chunks."""
    R, n = 1500, 6
    top = pi.make_chain(n, 3)
    ctx = lib.pamd_init(top, R, 500.0, 71, _opts(lib, resample_rule=3))
    try:
        cap = lib.pamd_population_size(ctx)[1]
        E = np.zeros(cap)
        E[:R] = -10.0
        E[3] = -3000.0  # weight ratio e^(0.01 * 2990): tau_3 ~ R
        lib.pamd_set_state(ctx, np.zeros((cap, n, 3)), np.zeros((cap, n, 3)), E)
        cnt, _ = lib.pamd_resample(ctx, 500.0, 480.0)
        _, W = orc.resample_weights(E[:R], 500.0, 480.0)
        ref = ov.poisson_counts(W, R, 71, 1)
        assert ref[3] > 1000
        np.testing.assert_array_equal(cnt[:R], ref)
    finally:
        lib.pamd_destroy(ctx)


def test_empty_population_is_reported(lib, orc):
    """R = 1 with Poisson copy numbers: a resampling index whose draw is zero
    (found with the oracle) empties the population."""
    top = pi.make_chain(5, 1)
    E1 = np.array([-3.0])
    _, W = orc.resample_weights(E1, 400.0, 390.0)
    ridx = next(i for i in range(1, 200) if ov.poisson_counts(W, 1, 13, i)[0] == 0)
    ctx = lib.pamd_init(top, 1, 400.0, 13, _opts(lib, resample_rule=3))
    try:
        cap = lib.pamd_population_size(ctx)[1]
        E = np.zeros(cap); E[0] = -3.0
        lib.pamd_set_state(ctx, np.zeros((cap, 5, 3)), np.zeros((cap, 5, 3)), E)
        lib.pamd_set_counters(ctx, 0, ridx - 1, 0.0)
        with pytest.raises(lib.PamdError) as ei:
            lib.pamd_resample(ctx, 400.0, 390.0)
        assert ei.value.code == lib.PAMD_EPOPSIZE
        assert lib.pamd_population_size(ctx)[0] == 0
    finally:
        lib.pamd_destroy(ctx)


def _runs_mean_and_se(runs, key, se):
    v = np.array([[o[key] for o in r] for r in runs])
    f = np.array([[o[se] for o in r] for r in runs])
    n = v.shape[0]
    return v.mean(0), np.maximum(v.std(0, ddof=1) / np.sqrt(n), np.sqrt((f ** 2).sum(0)) / n)


@pytest.mark.parametrize("rule", ["nearest", "poisson"])
def test_varsize_anneal_harmonic_closed_forms(lib, rule):
    code, _ = RULES[rule]
    n, kb = 6, 400.0
    top = pi.make_harmonic_chain(n, kb, 0.0)
    temps = pi.geometric_schedule(400.0, 200.0, 6)
    runs, sizes = [], []
    for k in range(8):
        ctx = lib.pamd_init(top, 4096, temps[0], 11 + 7 * k, _opts(lib, gamma_per_ps=5.0,
                                                                    resample_rule=code))
        try:
            lib.pamd_propagate(ctx, 2000, 0.002, temps[0])
            obs = lib.pamd_anneal(ctx, temps, 200, 0.002)
            runs.append(obs)
            sizes.append([o["R_live"] for o in obs])
            assert obs[-1]["R_live"] == lib.pamd_population_size(ctx)[0]
        finally:
            lib.pamd_destroy(ctx)
    sizes = np.array(sizes)
    assert np.all(sizes[:, 0] == 4096)
    assert np.all(np.abs(sizes - 4096) < 8 * 64)
    assert np.any(sizes[:, 1:] != 4096)  # the size does vary
    e, se = _runs_mean_and_se(runs, "e_pot", "e_pot_se")
    e_exact = 1.5 * (n - 1) * KB * temps
    assert np.all(np.abs(e - e_exact) <= 3 * se), (e - e_exact) / se
    f = np.array([[o["sum_lnQ"] for o in r] for r in runs])
    f_exact = 1.5 * (n - 1) * np.log(temps / temps[0])
    f_se = np.maximum(f.std(0, ddof=1) / np.sqrt(len(runs)), 1e-12)
    assert np.all(np.abs(f.mean(0) - f_exact) <= 3 * f_se + 1e-9), (f.mean(0) - f_exact) / f_se


@pytest.mark.parametrize("rule", ["nearest", "poisson"])
def test_varsize_anneal_statistical_parity(lib, orc, rule):
    """22-atom chain, R = 256, theta = 100, 10 geometric steps 1000 -> 400 K:
    eight anneals on each side, <E_pot>(T) and <R_g>(T) within 3 combined
    standard errors of the oracle's, and the mean population sizes close."""
    code, _ = RULES[rule]
    top = pi.make_chain(22, 1)
    temps = pi.geometric_schedule(1000.0, 400.0, 10)
    R, theta, dt, gamma = 256, 100, 0.001, 1.0
    seeds = [101 + 37 * k for k in range(8)]
    og = []
    for sd in seeds:
        ctx = lib.pamd_init(top, R, temps[0], sd, _opts(lib, gamma_per_ps=gamma, resample_rule=code))
        try:
            og.append(lib.pamd_anneal(ctx, temps, theta, dt))
        finally:
            lib.pamd_destroy(ctx)
    oo = [ov.anneal(top, R, temps, theta, dt, gamma, sd + 3, rule) for sd in seeds]
    for key, se in (("e_pot", "e_pot_se"), ("rg", "rg_se")):
        g, sg = _runs_mean_and_se(og, key, se)
        o, so = _runs_mean_and_se(oo, key, se)
        s = np.hypot(sg, so)
        assert np.all(np.abs(g - o) <= 3 * s), (key, (g - o) / s)
    ng = np.array([[o["R_live"] for o in r] for r in og], dtype=float)
    no = np.array([[o["R"] for o in r] for r in oo], dtype=float)
    s = np.hypot(ng.std(0, ddof=1), no.std(0, ddof=1)) / math.sqrt(len(seeds)) + 1e-9
    assert np.all(np.abs(ng.mean(0) - no.mean(0)) <= 3 * s + 1.0)
