"""GPU parity of the adaptive temperature step, the adaptive anneal and
systematic resampling, through the C-ABI, against oracle/adaptive.py.

Tolerances: the GPU evaluates the overlap in FP32 exponentials on E - min E
(relative error of the estimate ~1e-6) and stops its multisection at
~1e-6 of dbeta_final, so its dbeta is held to 1e-5 of dbeta_final of the
oracle's FP64 root and its overlap, re-evaluated by the oracle, to 5e-5 of
the target; systematic copy counts are integer work and bit-exact.
"""
import math

import numpy as np
import pytest

import pamd_inputs as pi

pytestmark = pytest.mark.gpu

KB = 0.008314462618


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_06016_gb300 import build, pamd
    import oracle as orc
    from oracle import adaptive as oa
    build.build()
    orc.build()
    pamd.load()
    return torch, pamd, orc, oa


def _check_step(oa, E, T_prev, T_final, alpha, T_gpu, a_gpu):
    beta = 1.0 / (KB * T_prev)
    d_final = 1.0 / (KB * T_final) - beta
    T_or, _ = oa.next_temperature(E, T_prev, T_final, alpha)
    d_gpu = 1.0 / (KB * T_gpu) - beta
    d_or = 1.0 / (KB * T_or) - beta
    assert abs(d_gpu - d_or) <= 1e-5 * d_final, (T_gpu, T_or)
    a = oa.overlap(E, d_gpu)
    assert abs(a - a_gpu) < 1e-5
    if T_gpu == T_final:
        assert a >= alpha - 5e-5
    else:
        assert abs(a - alpha) < 5e-5, (a, alpha)


@pytest.mark.parametrize("R,alpha", [(1, 0.5), (7, 0.5), (1000, 0.3), (4099, 0.5), (65536, 0.8),
                                     (1 << 20, 0.5)])
def test_overlap_temperature_matches_oracle(env, R, alpha):
    torch, pamd, _, oa = env
    rng = np.random.default_rng(R)
    E = rng.gamma(30.0, KB * 900.0, R) - 2000.0
    dev = torch.from_numpy(E).cuda()
    for T_final in (850.0, 600.0, 200.0):
        T, a = pamd.pamd_overlap_temperature(dev.data_ptr(), R, 900.0, T_final, alpha)
        _check_step(oa, E, 900.0, T_final, alpha, T, a)


def test_overlap_temperature_non_finite_energy(env):
    torch, pamd, _, _ = env
    E = torch.zeros(100, dtype=torch.float64, device="cuda")
    E[17] = float("nan")
    with pytest.raises(pamd.PamdError) as ei:
        pamd.pamd_overlap_temperature(E.data_ptr(), 100, 500.0, 300.0, 0.5)
    assert ei.value.code == pamd.PAMD_ENONFINITE
    # equal energies: every temperature overlaps fully, so the step goes to T_final
    E.fill_(-3.0)
    T, a = pamd.pamd_overlap_temperature(E.data_ptr(), 100, 500.0, 300.0, 0.99)
    assert T == 300.0 and a == 1.0


def test_next_temperature_of_a_population(env):
    torch, pamd, _, oa = env
    top = pi.make_chain(22, 1)
    ctx = pamd.pamd_init(top, 512, 800.0, 5)
    try:
        pamd.pamd_propagate(ctx, 200, 0.001, 800.0)
        E = pamd.pamd_get_state(ctx, False, False, True, False)[2]
        T, a = pamd.pamd_next_temperature(ctx, 800.0, 300.0, 0.6)
        _check_step(oa, E, 800.0, 300.0, 0.6, T, a)
        # the step does not change the population
        np.testing.assert_array_equal(pamd.pamd_get_state(ctx, False, False, True, False)[2], E)
    finally:
        pamd.pamd_destroy(ctx)


def test_adaptive_anneal_steps_meet_the_overlap_condition(env):
    torch, pamd, orc, oa = env
    top = pi.make_chain(22, 1)
    R, theta, dt, alpha, seed = 256, 100, 0.001, 0.5, 77
    rec = torch.empty((41, R), dtype=torch.float64, device="cuda")
    ctx = pamd.pamd_init(top, R, 1000.0, seed)
    try:
        pamd.pamd_record_energies(ctx, rec.data_ptr(), 41)
        obs, temps = pamd.pamd_anneal_adaptive(ctx, 1000.0, 300.0, alpha, theta, dt, 40)
    finally:
        pamd.pamd_destroy(ctx)
    n = len(temps)
    assert n >= 3 and np.all(np.diff(temps) < 0) and temps[-1] >= 300.0
    assert [o["T"] for o in obs] == list(temps)
    E = rec.cpu().numpy()[:n]
    for i in range(1, n):
        d = 1.0 / (KB * temps[i]) - 1.0 / (KB * temps[i - 1])
        a = oa.overlap(E[i - 1], d)
        if temps[i] == 300.0:
            assert a >= alpha - 5e-5
        else:
            assert abs(a - alpha) < 5e-5, (i, a)
    # statistics along the chosen schedule: four GPU and four oracle anneals
    # over it (independent seeds); per side the larger of the run-to-run
    # standard error and the pooled family-binned error
    runs_g, runs_o = [], []
    for k in range(4):
        c = pamd.pamd_init(top, R, temps[0], seed + 100 * k)
        try:
            runs_g.append(pamd.pamd_anneal(c, temps, theta, dt))
        finally:
            pamd.pamd_destroy(c)
        runs_o.append(orc.anneal(top, R, temps, theta, dt, 1.0, seed + 100 * k)[0])

    def mean_and_se(runs):
        v = np.array([[o["e_pot"] for o in r] for r in runs])
        f = np.array([[o["e_pot_se"] for o in r] for r in runs])
        return v.mean(0), np.maximum(v.std(0, ddof=1) / 2.0, np.sqrt((f ** 2).sum(0)) / 4.0)

    g, sg = mean_and_se(runs_g)
    o_, so = mean_and_se(runs_o)
    s = np.hypot(sg, so)
    assert np.all(np.abs(g - o_) <= 3 * s), (g - o_) / s


def test_adaptive_anneal_of_a_harmonic_chain_is_geometric(env):
    """The overlap of two Gamma(k) energy densities depends on T2/T1 only, so
    the schedule must be geometric with the ratio that solves the closed form."""
    from scipy.optimize import brentq
    from scipy.special import gammainc
    torch, pamd, _, _ = env
    n, kb = 6, 400.0
    k = 1.5 * (n - 1)

    def gamma_overlap(r):  # T2 / T1 = r
        Es = k * math.log(1.0 / r) / (1.0 / r - 1.0)
        return gammainc(k, Es) + 1.0 - gammainc(k, Es / r)

    alpha = 0.7
    r_exact = brentq(lambda r: gamma_overlap(r) - alpha, 1e-6, 1.0 - 1e-9)
    opts = pamd.pamd_options_default()
    opts.gamma_per_ps = 5.0
    ctx = pamd.pamd_init(pi.make_harmonic_chain(n, kb, 0.0), 8192, 400.0, 21, opts)
    try:
        obs, temps = pamd.pamd_anneal_adaptive(ctx, 400.0, 150.0, alpha, 200, 0.002, 40)
    finally:
        pamd.pamd_destroy(ctx)
    ratios = temps[1:] / temps[:-1]
    assert temps[-1] == 150.0
    assert np.all(np.abs(ratios[:-1] - r_exact) < 0.02), (ratios, r_exact)
    e = np.array([o["e_pot"] for o in obs]); se = np.array([o["e_pot_se"] for o in obs])
    assert np.all(np.abs(e - k * KB * temps) < 4 * se + 0.01 * k * KB * temps)
    # sum of ln Q: per step the estimate scatters by about sqrt(var w / R) / <w>
    # (0.01 here, times the correlation of resampled copies); a few steps
    f = np.array([o["sum_lnQ"] for o in obs])
    assert np.all(np.abs(f - k * np.log(temps / temps[0])) < 0.1), f - k * np.log(temps / temps[0])


@pytest.mark.parametrize("R", [1, 5, 1000, 4097, 1 << 18])
def test_systematic_copy_counts_bit_exact(env, R):
    torch, pamd, orc, oa = env
    top = pi.make_chain(13, 2)
    opts = pamd.pamd_options_default()
    opts.resample_rule = pamd.PAMD_RESAMPLE_SYSTEMATIC
    ctx = pamd.pamd_init(top, R, 900.0, 31, opts)
    try:
        pamd.pamd_propagate(ctx, 20, 0.001, 900.0)
        for i, (Tp, Tn) in enumerate([(900.0, 700.0), (700.0, 500.0)], start=1):
            E = pamd.pamd_get_state(ctx, False, False, True, False)[2]
            _, W = orc.resample_weights(E, Tp, Tn)
            cnt, _ = pamd.pamd_resample(ctx, Tp, Tn)
            want = oa.systematic_counts(W, 31, i)
            np.testing.assert_array_equal(cnt, want)
            pamd.pamd_propagate(ctx, 5, 0.001, Tn)
    finally:
        pamd.pamd_destroy(ctx)


def test_systematic_resampling_keeps_the_harmonic_closed_forms(env):
    torch, pamd, _, _ = env
    n, kb = 6, 400.0
    temps = pi.geometric_schedule(400.0, 200.0, 6)
    opts = pamd.pamd_options_default()
    opts.gamma_per_ps = 5.0
    opts.resample_rule = pamd.PAMD_RESAMPLE_SYSTEMATIC
    ctx = pamd.pamd_init(pi.make_harmonic_chain(n, kb, 0.0), 4096, temps[0], 11, opts)
    try:
        obs = pamd.pamd_anneal(ctx, temps, 200, 0.002)
    finally:
        pamd.pamd_destroy(ctx)
    e = np.array([o["e_pot"] for o in obs]); se = np.array([o["e_pot_se"] for o in obs])
    e_exact = 1.5 * (n - 1) * KB * temps
    assert np.all(np.abs(e - e_exact) < 4 * se + 0.005 * e_exact), (e - e_exact) / se
    f = np.array([o["sum_lnQ"] for o in obs])
    assert np.all(np.abs(f - 1.5 * (n - 1) * np.log(temps / temps[0])) < 0.05)


def test_adaptive_anneal_with_resampling_off(env):
    """The control run on an overlap-chosen schedule: no family is pruned and
    every step still meets the overlap condition on the recorded energies."""
    torch, pamd, _, oa = env
    top = pi.make_chain(22, 1)
    R, alpha = 128, 0.6
    rec = torch.empty((21, R), dtype=torch.float64, device="cuda")
    ctx = pamd.pamd_init(top, R, 900.0, 5)
    try:
        pamd.pamd_record_energies(ctx, rec.data_ptr(), 21)
        obs, temps = pamd.pamd_anneal_adaptive(ctx, 900.0, 400.0, alpha, 50, 0.001, 20, resample=False)
        fam = pamd.pamd_get_state(ctx, False, False, False, True)[3]
    finally:
        pamd.pamd_destroy(ctx)
    np.testing.assert_array_equal(fam, np.arange(R))
    assert all(o["n_families"] == R for o in obs)
    E = rec.cpu().numpy()
    for i in range(1, len(temps)):
        d = 1.0 / (KB * temps[i]) - 1.0 / (KB * temps[i - 1])
        a = oa.overlap(E[i - 1], d)
        assert (a >= alpha - 5e-5) if temps[i] == 400.0 else abs(a - alpha) < 5e-5
