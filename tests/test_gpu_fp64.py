"""All-FP64 mode (PAMD_PREC_FP64) against the FP64 oracle.

With every quantity in binary64 the GPU path matches the oracle to rounding:
forces to 1e-10 relative RMS, 10-step trajectories to 1e-10 nm (the noise
comes from the same Philox words; only libm and CUDA log/cos may differ in the
last ulp), copy counts bit-exact.  It is the precision reference of the
mixed FP32/FP64 kernels.
"""
import math

import numpy as np
import pytest

import pamd_inputs as pi

pytestmark = pytest.mark.gpu
KB = 0.008314462618


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
    o.precision = lib.PAMD_PREC_FP64
    for k, v in kw.items():
        setattr(o, k, v)
    return o


@pytest.mark.parametrize("n", [1, 5, 22, 75, 200])
def test_fp64_forces(lib, orc, n):
    top = pi.make_chain(n, 300 + n)
    top.dih_phase = np.linspace(0.3, 1.9, len(top.dih_phase))
    R = 5
    x = pi.perturbed_positions(top, R, 0.01, n)
    ctx = lib.pamd_init(top, R, 300.0, 1, _opts(lib))
    try:
        lib.pamd_set_state(ctx, x, np.zeros_like(x))
        fg, eg = lib.pamd_forces(ctx)
    finally:
        lib.pamd_destroy(ctx)
    t = orc.Topo(top)
    for k in range(R):
        e, f, terms = orc.energy_forces(t, x[k])
        rms = math.sqrt(np.mean(f ** 2)) if n > 1 else 1.0
        assert math.sqrt(np.mean((fg[k] - f) ** 2)) <= 1e-10 * max(rms, 1e-12)
        assert abs(eg[k] - e) <= 1e-10 * max(np.abs(terms).sum(), 1e-12)


def test_fp64_trajectory_and_init(lib, orc):
    top = pi.make_chain(22, 7)
    R, T, dt, gamma, seed = 6, 500.0, 0.001, 1.0, 99
    ctx = lib.pamd_init(top, R, T, seed, _opts(lib, gamma_per_ps=gamma))
    try:
        x0, v0, _, fam = lib.pamd_get_state(ctx)
        xo, vo, fo = orc.init(top, R, T, seed)
        assert np.abs(x0 - xo).max() < 1e-13 and np.abs(v0 - vo).max() < 1e-12
        np.testing.assert_array_equal(fam, fo)
        for s in range(10):
            lib.pamd_propagate(ctx, 1, dt, T)
            xg, vg, eg, _ = lib.pamd_get_state(ctx)
            xo, vo, eo = orc.propagate(top, xo, vo, 1, dt, T, gamma, seed, s)
            assert np.abs(xg - xo).max() < 1e-10, (s, np.abs(xg - xo).max())
        assert np.abs(eg - eo).max() < 1e-8
    finally:
        lib.pamd_destroy(ctx)


def test_fp64_resample_and_gather(lib, orc):
    top = pi.make_chain(9, 2)
    R, seed = 1500, 12
    x = pi.perturbed_positions(top, R, 0.02, 5)
    v = pi.gaussian_velocities(R, 9, 0.5, 6)
    E = pi.random_energies(R, -50.0, 20.0, 8)
    fam = np.arange(R, dtype=np.int32)
    ctx = lib.pamd_init(top, R, 700.0, seed, _opts(lib))
    try:
        lib.pamd_set_state(ctx, x, v, E, fam)
        cnt, lnq = lib.pamd_resample(ctx, 700.0, 650.0)
        xg, vg, eg, fg = lib.pamd_get_state(ctx)
    finally:
        lib.pamd_destroy(ctx)
    lnq_o, W = orc.resample_weights(E, 700.0, 650.0)
    cnt_o = orc.multinomial_counts(W, seed, 1)
    np.testing.assert_array_equal(cnt, cnt_o)
    xo, vo, fo, eo = orc.gather(top, cnt_o, x, v, fam, E, math.sqrt(650.0 / 700.0))
    np.testing.assert_array_equal(fg, fo)
    assert np.abs(xg - xo).max() < 1e-12
    assert np.abs(vg - vo).max() < 1e-13


def test_fp64_anneal_graph_and_oracle(lib, orc):
    top = pi.make_chain(12, 4)
    temps = pi.geometric_schedule(800.0, 600.0, 3)
    R, theta, dt, seed = 64, 10, 0.001, 5
    ctx = lib.pamd_init(top, R, temps[0], seed, _opts(lib))
    try:
        og = lib.pamd_anneal(ctx, temps, theta, dt)
    finally:
        lib.pamd_destroy(ctx)
    oo, *_ = orc.anneal(top, R, temps, theta, dt, 1.0, seed)
    # same FP64 arithmetic and random numbers: the whole anneal agrees closely
    for a, b in zip(og, oo):
        assert abs(a["e_pot"] - b["e_pot"]) < 1e-6 * max(1.0, abs(b["e_pot"]))
        assert abs(a["sum_lnQ"] - b["sum_lnQ"]) < 1e-9
        assert a["n_families"] == b["n_families"]
