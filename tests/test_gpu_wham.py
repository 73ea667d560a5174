"""GPU parity of the multiple-histogram reweighting (pamd_wham) and of the
energy record of pamd_anneal, through the C-ABI.

Tolerances: histograms bit-exact (integer counts from the same FP64 bin
arithmetic); ln Z, ln g and the reweighted averages within 1e-10 of the FP64
oracle after the same number of sweeps (same operations, only the order of
the sums of exponentials differs); the recorded energies bit-exact against the
step-by-step calls.
"""
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
    from oracle import wham as ow
    build.build()
    pamd.load()
    return torch, pamd, ow


def _samples(seed, T, R, d=15, shift=-40.0, bad=True):
    rng = np.random.default_rng(seed)
    E = np.stack([rng.gamma(d / 2, KB * t, R) + shift for t in T])
    if bad:
        E[0, 3] = np.nan
        E[-1, 5] = np.inf
        E[1 % len(T), 7] = -np.inf
    return E


def _run_both(env, E, T, n_bins, **kw):
    torch, pamd, ow = env
    dev = torch.from_numpy(np.ascontiguousarray(E)).cuda()
    g = pamd.pamd_wham(dev.data_ptr(), E.shape[0], E.shape[1], T, n_bins, want_hist=True, **kw)
    torch.cuda.synchronize()
    e_range = kw.pop("e_range", None)
    lo, hi = (None, None) if e_range is None else e_range
    o = ow.wham(E, T, n_bins, lo, hi, kw.get("lnZ_init"), kw.get("max_iter", 100), kw.get("tol", 1e-10),
                kw.get("T_eval"))
    return g, o


def _compare(g, o, n_eval=0):
    np.testing.assert_array_equal(g["hist"], o["hist"])
    assert g["e_min"] == o["e_min"] and g["bin_width"] == o["bin_width"]
    assert g["iterations"] == o["iterations"]
    np.testing.assert_allclose(g["lnZ"], o["lnZ"], rtol=0, atol=1e-10)
    fin = np.isfinite(o["ln_g"])
    np.testing.assert_array_equal(np.isfinite(g["ln_g"]), fin)
    np.testing.assert_allclose(g["ln_g"][fin], o["ln_g"][fin], rtol=0, atol=1e-10)
    if n_eval:
        np.testing.assert_allclose(g["lnZ_eval"], o["lnZ_eval"], rtol=0, atol=1e-10)
        np.testing.assert_allclose(g["e_mean_eval"], o["e_mean_eval"], rtol=1e-12, atol=1e-10)
        np.testing.assert_allclose(g["e_var_eval"], o["e_var_eval"], rtol=1e-10)


@pytest.mark.parametrize("n_bins,R,n_temps", [(300, 5000, 9), (1, 17, 3), (257, 1, 4), (20000, 30000, 5),
                                              (12288, 4099, 2), (4096, 3001, 3), (4097, 3001, 3)])
def test_wham_matches_oracle_at_fixed_sweeps(env, n_bins, R, n_temps):
    T = np.geomspace(500.0, 250.0, n_temps)
    E = _samples(n_bins + R, T, R, bad=R >= 8)
    Te = [480.0, 333.0, 251.0]
    g, o = _run_both(env, E, T, n_bins, max_iter=40, tol=0.0, T_eval=Te)
    _compare(g, o, len(Te))


def test_wham_given_range_and_start_values(env):
    T = np.geomspace(600.0, 300.0, 6)
    E = _samples(3, T, 8000, bad=False)
    # the closed form plus a constant (the gauge removes the constant)
    z0 = 0.5 * 15 * np.log(T / T[0]) + 40.0 / (KB * T) + 3.0
    g, o = _run_both(env, E, T, 500, e_range=(-35.0, 10.0), lnZ_init=z0, max_iter=7, tol=0.0,
                     T_eval=[450.0])
    _compare(g, o, 1)
    # samples outside the given range are not counted
    assert g["hist"].sum() < E.size


def test_wham_converges_with_the_oracle(env):
    T = np.geomspace(400.0, 200.0, 8)
    E = _samples(11, T, 20000, bad=False)
    g, o = _run_both(env, E, T, 400, max_iter=4000, tol=1e-11)
    assert o["iterations"] < 4000 and abs(g["iterations"] - o["iterations"]) <= 1
    np.testing.assert_allclose(g["lnZ"], o["lnZ"], rtol=0, atol=1e-9)
    # Gamma(d/2, k_B T) energies shifted by -40: ln Z(T) gains +40 / k_B T
    d, beta = 15, 1.0 / (KB * T)
    exact = 0.5 * d * np.log(T / T[0]) + 40.0 * (beta - beta[0])
    assert np.max(np.abs(g["lnZ"] - exact)) < 0.05, g["lnZ"] - exact


def test_wham_degenerate_and_error_cases(env):
    torch, pamd, ow = env
    E = np.full((2, 10), 7.25)
    g, o = _run_both(env, E, np.array([300.0, 200.0]), 4, max_iter=3, tol=0.0)
    _compare(g, o)
    assert g["e_min"] == 7.25 and g["bin_width"] == 0.25
    dev = torch.from_numpy(E).cuda()
    with pytest.raises(pamd.PamdError) as ei:
        pamd.pamd_wham(dev.data_ptr(), 2, 10, [300.0, 200.0], 4, e_range=(100.0, 200.0))
    assert ei.value.code == pamd.PAMD_EINVAL
    nan = torch.full((1, 5), float("nan"), dtype=torch.float64, device="cuda")
    with pytest.raises(pamd.PamdError):
        pamd.pamd_wham(nan.data_ptr(), 1, 5, [300.0], 4)
    # zero sweeps: the start values (shifted), change reported as infinite
    g = pamd.pamd_wham(dev.data_ptr(), 2, 10, [300.0, 200.0], 4, lnZ_init=[1.0, 2.5], max_iter=0)
    assert g["iterations"] == 0 and np.isinf(g["max_delta"])
    np.testing.assert_array_equal(g["lnZ"], [0.0, 1.5])


def test_anneal_energy_record_matches_stepwise_calls(env):
    torch, pamd, _ = env
    top = pi.make_chain(22, 1)
    temps = pi.geometric_schedule(900.0, 500.0, 5)
    R, theta, dt = 256, 20, 0.001
    rec = torch.full((len(temps) + 2, R), -1.0, dtype=torch.float64, device="cuda")
    a = pamd.pamd_init(top, R, temps[0], 9)
    b = pamd.pamd_init(top, R, temps[0], 9)
    try:
        pamd.pamd_record_energies(a, rec.data_ptr(), len(temps) + 2)
        pamd.pamd_anneal(a, temps, theta, dt)
        rows = []
        pamd.pamd_propagate(b, theta, dt, temps[0])
        rows.append(pamd.pamd_get_state(b, False, False, True, False)[2])
        for i in range(1, len(temps)):
            pamd.pamd_resample(b, temps[i - 1], temps[i], want_copies=False)
            pamd.pamd_propagate(b, theta, dt, temps[i])
            rows.append(pamd.pamd_get_state(b, False, False, True, False)[2])
        got = rec.cpu().numpy()
        np.testing.assert_array_equal(got[: len(temps)], np.array(rows))
        assert np.all(got[len(temps):] == -1.0)  # rows beyond K + 1 are untouched
        # recording off: a second anneal leaves the record as it was
        pamd.pamd_record_energies(a, 0, 0)
        pamd.pamd_anneal(a, temps, theta, dt)
        np.testing.assert_array_equal(rec.cpu().numpy(), got)
    finally:
        pamd.pamd_destroy(a)
        pamd.pamd_destroy(b)


def test_harmonic_chain_anneal_then_wham_gives_the_closed_forms(env):
    """Bonds-only chain with r0 = 0: ln Z(T_i) - ln Z(T_0) = (3/2)(N-1) ln(T_i/T_0)
    and <E>(T) = (3/2)(N-1) k_B T; WHAM seeded with the running sum of ln Q."""
    torch, pamd, _ = env
    n, kb = 6, 400.0
    top = pi.make_harmonic_chain(n, kb, 0.0)
    temps = pi.geometric_schedule(400.0, 200.0, 6)
    R = 4096
    opts = pamd.pamd_options_default()
    opts.gamma_per_ps = 5.0
    ctx = pamd.pamd_init(top, R, temps[0], 11, opts)
    rec = torch.empty((len(temps), R), dtype=torch.float64, device="cuda")
    try:
        pamd.pamd_record_energies(ctx, rec.data_ptr(), len(temps))
        obs = pamd.pamd_anneal(ctx, temps, 200, 0.002)
    finally:
        pamd.pamd_destroy(ctx)
    z0 = np.array([o["sum_lnQ"] for o in obs])
    T_eval = np.array([350.0, 300.0, 250.0])
    g = pamd.pamd_wham(rec.data_ptr(), len(temps), R, temps, 200, lnZ_init=z0, max_iter=2000, tol=1e-11,
                       T_eval=T_eval)
    d = 3 * (n - 1)
    exact = 0.5 * d * np.log(temps / temps[0])
    assert np.max(np.abs(g["lnZ"] - exact)) < 0.05, g["lnZ"] - exact
    np.testing.assert_allclose(g["e_mean_eval"], 0.5 * d * KB * T_eval, rtol=0.02)


def test_wham_range_edges_and_signed_zero(env):
    """Samples at and next to the range ends, signed zeros and denormals are
    counted exactly as the IEEE comparisons of the definition count them."""
    T = np.array([300.0, 250.0])
    edge = [0.0, -0.0, 5e-324, -5e-324, 10.0, np.nextafter(10.0, 20.0), np.nextafter(10.0, 0.0),
            np.nextafter(0.0, -1.0), 2.5, 7.5, np.nan, -np.inf, np.inf]
    E = np.array([edge, edge[::-1]])
    g, o = _run_both(env, E, T, 4, e_range=(0.0, 10.0), max_iter=2, tol=0.0)
    _compare(g, o)
    assert g["hist"].sum() == 2 * 7
    g, o = _run_both(env, E, T, 3, e_range=(-0.0, 10.0), max_iter=2, tol=0.0)
    _compare(g, o)
