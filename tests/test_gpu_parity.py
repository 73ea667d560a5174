"""GPU parity: the CUDA library (through the C-ABI) against the FP64 oracle.

Tolerances (from the method's precision contract):
  * forces: relative RMS error <= 1e-5 per replica (FP32 forces);
  * energies: |dE| <= 1e-5 * sum of the magnitudes of the energy terms
    (FP32 terms summed in FP64);
  * trajectories: every position within 1e-4 nm of the oracle after each of
    10 BAOAB steps from the same state and the same Philox stream;
  * copy counts: bit-exact, given the same energies;
  * ln Q: 1e-12 absolute (FP64 log-sum-exp, different summation order);
  * population averages of an anneal: within 3 combined standard errors.
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


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _opts(lib, **kw):
    o = lib.pamd_options_default()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _oracle_forces(orc, top, x):
    t = orc.Topo(top)
    F = np.zeros_like(x)
    E = np.zeros(x.shape[0])
    scale = np.zeros(x.shape[0])
    for k in range(x.shape[0]):
        e, f, terms = orc.energy_forces(t, x[k])
        F[k], E[k] = f, e
        # magnitude of the individual contributions, for the energy tolerance
        scale[k] = np.abs(terms).sum()
    return F, E, scale


FORCE_CASES = [(1, 0), (2, 0), (3, 0), (4, 0), (5, 0), (13, 0), (22, 0), (22, 8), (22, 16),
               (31, 0), (33, 0), (64, 0), (75, 0), (75, 32), (129, 0), (200, 0), (256, 0)]


def _init_arith(lib, top, R, T, seed, arith, **kw):
    """Context with the scalar or the packed pair arithmetic; shapes the
    packed kernel does not serve (fewer than 3 atoms per lane) are skipped."""
    pa = lib.PAMD_PAIRS_SCALAR if arith == "scalar" else lib.PAMD_PAIRS_PACKED
    try:
        return lib.pamd_init(top, R, T, seed, _opts(lib, pair_arith=pa, **kw))
    except lib.PamdError as e:
        if arith == "packed" and e.code == lib.PAMD_EUNSUPPORTED:
            pytest.skip("packed pair arithmetic does not apply to this shape")
        raise


@pytest.mark.parametrize("arith", ["scalar", "packed"])
@pytest.mark.parametrize("n,lanes", FORCE_CASES)
def test_forces_and_energies(lib, orc, n, lanes, arith):
    top = pi.make_chain(n, 100 + n)
    top.dih_phase = np.linspace(0.2, 1.7, len(top.dih_phase))  # exercise the torsion sign
    R = 7
    x = f32(pi.perturbed_positions(top, R, 0.01, n))
    v = np.zeros_like(x)
    ctx = _init_arith(lib, top, R, 300.0, 1, arith, lanes_per_replica=lanes)
    try:
        lib.pamd_set_state(ctx, x, v)
        fg, eg = lib.pamd_forces(ctx)
    finally:
        lib.pamd_destroy(ctx)
    fo, eo, scale = _oracle_forces(orc, top, x)
    for k in range(R):
        rms = math.sqrt(np.mean(fo[k] ** 2))
        if rms > 0:
            assert math.sqrt(np.mean((fg[k] - fo[k]) ** 2)) <= 1e-5 * rms, (k, n)
        assert abs(eg[k] - eo[k]) <= 1e-5 * max(scale[k], 1e-3), (k, eg[k], eo[k])


# Packed FP32x2 pair arithmetic: every atoms-per-lane count 3..8, odd and
# even lane counts (the even ones halve the antipodal tile), lane counts that
# leave idle lanes, padding atoms, and R not a multiple of the replicas per
# block (a ragged last block).
PACKED_CASES = [(75, 25), (75, 19), (75, 15), (75, 13), (75, 11), (75, 10), (22, 8), (22, 6),
                (22, 4), (22, 3), (40, 8), (9, 3), (200, 29), (256, 32)]


@pytest.mark.parametrize("n,lanes", PACKED_CASES)
def test_packed_kernel_forces(lib, orc, n, lanes):
    top = pi.make_chain(n, 300 + n)
    top.dih_phase = np.linspace(0.3, 2.1, len(top.dih_phase))
    R = 11
    x = f32(pi.perturbed_positions(top, R, 0.01, n + 3))
    ctx = lib.pamd_init(top, R, 300.0, 1, _opts(lib, lanes_per_replica=lanes,
                                               pair_arith=lib.PAMD_PAIRS_PACKED))
    try:
        shape = lib.pamd_get_shape(ctx)
        assert shape["pair_arith"] == lib.PAMD_PAIRS_PACKED and shape["lanes_per_replica"] == lanes
        lib.pamd_set_state(ctx, x, np.zeros_like(x))
        fg, eg = lib.pamd_forces(ctx)
    finally:
        lib.pamd_destroy(ctx)
    fo, eo, scale = _oracle_forces(orc, top, x)
    for k in range(R):
        rms = math.sqrt(np.mean(fo[k] ** 2))
        assert math.sqrt(np.mean((fg[k] - fo[k]) ** 2)) <= 1e-5 * rms, (k, n)
        assert abs(eg[k] - eo[k]) <= 1e-5 * scale[k], (k, eg[k], eo[k])


@pytest.mark.parametrize("n,lanes,R", [(75, 15, 5), (75, 10, 3), (22, 6, 7), (40, 8, 9)])
def test_packed_kernel_trajectory(lib, orc, n, lanes, R):
    top = pi.make_chain(n, 7)
    T, dt, gamma, seed = 400.0, 0.001, 1.0, 4242
    x = f32(pi.perturbed_positions(top, R, 0.005, 1))
    x = f32(x - x.mean(axis=1, keepdims=True))
    v = f32(pi.gaussian_velocities(R, n, math.sqrt(KB * T / 12.0), 2))
    ctx = lib.pamd_init(top, R, T, seed, _opts(lib, gamma_per_ps=gamma, lanes_per_replica=lanes,
                                                pair_arith=lib.PAMD_PAIRS_PACKED))
    try:
        assert lib.pamd_get_shape(ctx)["pair_arith"] == lib.PAMD_PAIRS_PACKED
        lib.pamd_set_state(ctx, x, v)
        xo, vo = x.copy(), v.copy()
        for s in range(10):
            lib.pamd_propagate(ctx, 1, dt, T)
            xg, vg, eg, _ = lib.pamd_get_state(ctx)
            xo, vo, eo = orc.propagate(top, xo, vo, 1, dt, T, gamma, seed, s)
            assert np.abs(xg - xo).max() < 1e-4, (s, np.abs(xg - xo).max())
        assert np.abs(vg - vo).max() < 1e-2 * np.abs(vo).max()
        assert np.abs(eg - eo).max() < 1e-4 * max(np.abs(eo).max(), 1.0)
        # ten steps in one launch: the same trajectory as ten launches of one step
        lib.pamd_set_state(ctx, x, v)
        lib.pamd_set_counters(ctx, 0, 0, 0.0)
        lib.pamd_propagate(ctx, 10, dt, T)
        x10, v10, _, _ = lib.pamd_get_state(ctx)
        assert np.abs(x10 - xo).max() < 1e-4
    finally:
        lib.pamd_destroy(ctx)


PAIRED_CASES = [(13, 7, 6), (13, 7, 5), (22, 8, 7), (75, 25, 4), (75, 25, 3), (75, 19, 2),
                (40, 20, 5)]


@pytest.mark.parametrize("n,lanes,R", PAIRED_CASES)
def test_paired_kernel_forces(lib, orc, n, lanes, R):
    """Two replicas per lane group (packed FP32x2), including an odd R whose
    last group runs one replica twice."""
    top = pi.make_chain(n, 200 + n)
    top.dih_phase = np.linspace(0.2, 1.7, len(top.dih_phase))
    x = f32(pi.perturbed_positions(top, R, 0.01, n + 1))
    ctx = lib.pamd_init(top, R, 300.0, 1, _opts(lib, lanes_per_replica=lanes, replicas_per_lane=2))
    try:
        assert lib.pamd_info(ctx)["replicas_per_block"] % 2 == 0
        lib.pamd_set_state(ctx, x, np.zeros_like(x))
        fg, eg = lib.pamd_forces(ctx)
    finally:
        lib.pamd_destroy(ctx)
    fo, eo, scale = _oracle_forces(orc, top, x)
    for k in range(R):
        rms = math.sqrt(np.mean(fo[k] ** 2))
        assert math.sqrt(np.mean((fg[k] - fo[k]) ** 2)) <= 1e-5 * rms, (k, n)
        assert abs(eg[k] - eo[k]) <= 1e-5 * scale[k], (k, eg[k], eo[k])


@pytest.mark.parametrize("n,lanes,R", [(22, 8, 5), (75, 25, 3)])
def test_paired_kernel_trajectory(lib, orc, n, lanes, R):
    top = pi.make_chain(n, 7)
    T, dt, gamma, seed = 400.0, 0.001, 1.0, 4242
    x = f32(pi.perturbed_positions(top, R, 0.005, 1))
    x = f32(x - x.mean(axis=1, keepdims=True))
    v = f32(pi.gaussian_velocities(R, n, math.sqrt(KB * T / 12.0), 2))
    ctx = lib.pamd_init(top, R, T, seed, _opts(lib, gamma_per_ps=gamma, lanes_per_replica=lanes,
                                                replicas_per_lane=2))
    try:
        lib.pamd_set_state(ctx, x, v)
        xo, vo = x.copy(), v.copy()
        for s in range(10):
            lib.pamd_propagate(ctx, 1, dt, T)
            xg, vg, eg, _ = lib.pamd_get_state(ctx)
            xo, vo, eo = orc.propagate(top, xo, vo, 1, dt, T, gamma, seed, s)
            assert np.abs(xg - xo).max() < 1e-4, (s, np.abs(xg - xo).max())
        assert np.abs(eg - eo).max() < 1e-4 * max(np.abs(eo).max(), 1.0)
    finally:
        lib.pamd_destroy(ctx)


def _runs_mean_and_se(runs, key, se):
    """Mean over independent anneals per temperature, with the larger of the
    run-to-run standard error and the pooled family-binned error (a single
    small population ends with few families, whose binned error understates
    the spread of its means)."""
    v = np.array([[o[key] for o in r] for r in runs])
    f = np.array([[o[se] for o in r] for r in runs])
    n = v.shape[0]
    return v.mean(0), np.maximum(v.std(0, ddof=1) / np.sqrt(n), np.sqrt((f ** 2).sum(0)) / n)


def test_paired_and_single_kernels_agree_statistically(lib):
    """The two-replica kernel and the single-replica kernel run the same
    anneals (eight seeds each): the FP32 rounding differs, so the averages
    are compared within 3 combined standard errors."""
    top = pi.make_chain(22, 1)
    temps = pi.geometric_schedule(1000.0, 500.0, 6)
    runs = {1: [], 2: []}
    for rpl in (1, 2):
        for k in range(8):
            ctx = lib.pamd_init(top, 512, temps[0], 9 + 101 * k,
                                _opts(lib, lanes_per_replica=8, replicas_per_lane=rpl))
            try:
                runs[rpl].append(lib.pamd_anneal(ctx, temps, 50, 0.001))
            finally:
                lib.pamd_destroy(ctx)
    for key, se in (("e_pot", "e_pot_se"), ("rg", "rg_se")):
        a, sa = _runs_mean_and_se(runs[1], key, se)
        b, sb = _runs_mean_and_se(runs[2], key, se)
        assert np.all(np.abs(a - b) <= 3 * np.hypot(sa, sb)), (key, (a - b) / np.hypot(sa, sb))


@pytest.mark.parametrize("arith", ["scalar", "packed"])
@pytest.mark.parametrize("n,lanes", [(75, 15), (40, 8), (23, 5)])
def test_forces_chain_with_far_exclusions(lib, orc, n, lanes, arith):
    """A chain in index order (chain layout) with extra exclusions between
    distant atoms: masked pairs in ring tiles beyond the first, which the
    kernels must evaluate with the masked code."""
    top = pi.make_chain(n, 6)
    far = [(0, n - 1), (2, n // 2), (n // 3, n - 4), (1, 9)]
    top.excl = np.concatenate([np.asarray(top.excl, np.int32).reshape(-1, 2),
                               np.asarray(far, np.int32)]).astype(np.int32)
    R = 4
    x = f32(pi.perturbed_positions(top, R, 0.01, 3))
    ctx = _init_arith(lib, top, R, 300.0, 1, arith, lanes_per_replica=lanes)
    try:
        lib.pamd_set_state(ctx, x, np.zeros_like(x))
        fg, eg = lib.pamd_forces(ctx)
    finally:
        lib.pamd_destroy(ctx)
    fo, eo, scale = _oracle_forces(orc, top, x)
    for k in range(R):
        rms = math.sqrt(np.mean(fo[k] ** 2))
        assert math.sqrt(np.mean((fg[k] - fo[k]) ** 2)) <= 1e-5 * rms
        assert abs(eg[k] - eo[k]) <= 1e-5 * scale[k]


def test_default_pair_arithmetic(lib):
    """PAMD_PAIRS_AUTO starts with the packed arithmetic where its layout
    applies (a chain with 3..8 atoms per lane, mixed precision, one replica
    per lane group) and with the scalar one elsewhere."""
    def arith(top, **kw):
        ctx = lib.pamd_init(top, 64, 300.0, 1, _opts(lib, **kw))
        try:
            return lib.pamd_get_shape(ctx)["pair_arith"]
        finally:
            lib.pamd_destroy(ctx)
    chain = pi.make_chain(75, 2)
    assert arith(chain) == lib.PAMD_PAIRS_PACKED
    assert arith(chain, lanes_per_replica=15) == lib.PAMD_PAIRS_PACKED
    assert arith(pi.make_chain(40, 2), lanes_per_replica=20) == lib.PAMD_PAIRS_SCALAR  # 2 atoms per lane
    assert arith(chain, replicas_per_lane=2, lanes_per_replica=25) == lib.PAMD_PAIRS_SCALAR
    assert arith(pi.make_chain(8, 2), lanes_per_replica=8) == lib.PAMD_PAIRS_SCALAR  # 1 atom per lane
    relabelled = pi.make_chain(40, 5)
    perm = np.random.default_rng(3).permutation(40)
    for name in ("bond", "angle", "dihedral", "excl", "pair14"):
        setattr(relabelled, name, perm[getattr(relabelled, name)].astype(np.int32))
    assert arith(relabelled) == lib.PAMD_PAIRS_SCALAR


@pytest.mark.parametrize("n", [13, 40, 75])
def test_forces_relabelled_chain(lib, orc, n):
    """Atoms of a chain relabelled at random: the bonded terms are no longer a
    chain in index order and exclusions fall in every tile (generic path)."""
    base = pi.make_chain(n, 5)
    perm = np.random.default_rng(n).permutation(n)   # new index of old atom i
    inv = np.argsort(perm)
    top = pi.make_chain(n, 5)
    for name in ("mass", "charge", "sigma", "epsilon"):
        setattr(top, name, getattr(base, name)[inv])
    top.x0 = base.x0[inv]
    for name in ("bond", "angle", "dihedral", "excl", "pair14"):
        setattr(top, name, perm[getattr(base, name)].astype(np.int32))
    R = 4
    x = f32(pi.perturbed_positions(top, R, 0.01, 9))
    paired = 2 if n in (13, 75) else 1   # generic path of both kernel families
    lanes = {13: 5, 40: 0, 75: 25}[n]
    ctx = lib.pamd_init(top, R, 300.0, 1, _opts(lib, lanes_per_replica=lanes, replicas_per_lane=paired))
    try:
        lib.pamd_set_state(ctx, x, np.zeros_like(x))
        fg, eg = lib.pamd_forces(ctx)
    finally:
        lib.pamd_destroy(ctx)
    fo, eo, scale = _oracle_forces(orc, top, x)
    for k in range(R):
        rms = math.sqrt(np.mean(fo[k] ** 2))
        assert math.sqrt(np.mean((fg[k] - fo[k]) ** 2)) <= 1e-5 * rms
        assert abs(eg[k] - eo[k]) <= 1e-5 * scale[k]


def test_forces_excluded_overlapping_pairs(lib, orc):
    # bonds-only chain: every pair excluded, atoms may sit on top of each other
    top = pi.make_harmonic_chain(9, 400.0, 0.0, seed=3)
    R = 5
    x = f32(pi.perturbed_positions(top, R, 0.05, 2))
    x[0, 3] = x[0, 5]  # coincident non-bonded (excluded) atoms
    ctx = lib.pamd_init(top, R, 300.0, 1)
    try:
        lib.pamd_set_state(ctx, x, np.zeros_like(x))
        fg, eg = lib.pamd_forces(ctx)
    finally:
        lib.pamd_destroy(ctx)
    fo, eo, _ = _oracle_forces(orc, top, x)
    assert np.all(np.isfinite(fg)) and np.all(np.isfinite(eg))
    np.testing.assert_allclose(fg, fo, rtol=1e-5, atol=1e-4)
    np.testing.assert_allclose(eg, eo, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("arith", ["scalar", "packed"])
@pytest.mark.parametrize("n,R", [(22, 5), (75, 3), (200, 2), (7, 40)])
def test_ten_step_trajectory(lib, orc, n, R, arith):
    top = pi.make_chain(n, 7)
    T, dt, gamma, seed = 400.0, 0.001, 1.0, 4242
    x = f32(pi.perturbed_positions(top, R, 0.005, 1))
    x -= x.mean(axis=1, keepdims=True)
    x = f32(x)
    v = f32(pi.gaussian_velocities(R, n, math.sqrt(KB * T / 12.0), 2))
    ctx = _init_arith(lib, top, R, T, seed, arith, gamma_per_ps=gamma)
    try:
        lib.pamd_set_state(ctx, x, v)
        xo, vo = x.copy(), v.copy()
        for s in range(10):
            lib.pamd_propagate(ctx, 1, dt, T)
            xg, vg, eg, _ = lib.pamd_get_state(ctx)
            xo, vo, eo = orc.propagate(top, xo, vo, 1, dt, T, gamma, seed, s)
            assert np.abs(xg - xo).max() < 1e-4, (s, np.abs(xg - xo).max())
        assert np.abs(vg - vo).max() < 1e-2 * np.abs(vo).max()
        scale = max(np.abs(eo).max(), 1.0)
        assert np.abs(eg - eo).max() < 1e-4 * scale
    finally:
        lib.pamd_destroy(ctx)


def test_init_matches_oracle(lib, orc):
    top = pi.make_chain(22, 3)
    ctx = lib.pamd_init(top, 300, 800.0, 77)
    try:
        xg, vg, _, fam = lib.pamd_get_state(ctx)
    finally:
        lib.pamd_destroy(ctx)
    xo, vo, fo = orc.init(top, 300, 800.0, 77)
    np.testing.assert_array_equal(fam, fo)
    assert np.abs(xg - xo).max() < 1e-6
    assert np.abs(vg - vo).max() < 1e-5 * np.abs(vo).max()


RESAMPLE_CASES = [(1, 100.0), (2, 30.0), (3, 30.0), (1000, 30.0), (1025, 5.0), (4097, 60.0),
                  (3000, 1e5), (2048, 0.0)]


@pytest.mark.parametrize("R,spread", RESAMPLE_CASES)
def test_resample_bit_exact(lib, orc, R, spread):
    top = pi.make_chain(9, 2)
    seed = 99 + R
    x = f32(pi.perturbed_positions(top, R, 0.02, 5))
    v = f32(pi.gaussian_velocities(R, 9, 0.5, 6))
    E = pi.random_energies(R, -50.0, spread, 8)
    fam = np.arange(R, dtype=np.int32)[::-1].copy()
    Tp, Tn = 700.0, 640.0
    ctx = lib.pamd_init(top, R, Tp, seed)
    try:
        lib.pamd_set_state(ctx, x, v, E, fam)
        cnt, lnq = lib.pamd_resample(ctx, Tp, Tn)
        xg, vg, eg, fg = lib.pamd_get_state(ctx)
        obs = lib.pamd_observables(ctx, Tn)
    finally:
        lib.pamd_destroy(ctx)
    lnq_o, W = orc.resample_weights(E, Tp, Tn)
    cnt_o = orc.multinomial_counts(W, seed, 1)
    np.testing.assert_array_equal(cnt, cnt_o)
    assert cnt.sum() == R
    assert abs(lnq - lnq_o) <= 1e-12 * max(1.0, abs(lnq_o))
    xo, vo, fo, eo = orc.gather(top, cnt_o, x, v, fam, E, math.sqrt(Tn / Tp))
    np.testing.assert_array_equal(fg, fo)
    np.testing.assert_array_equal(eg, eo)
    assert np.abs(xg - xo).max() < 2e-6
    assert np.abs(vg - vo).max() <= 1e-6 * max(np.abs(vo).max(), 1e-30)
    assert obs["max_copies"] == cnt_o.max()
    assert abs(obs["lnQ"] - lnq_o) <= 1e-12 * max(1.0, abs(lnq_o))


# Gather of molecules whose state spans several float4 passes of a warp:
# 75 atoms (456 floats = 114 float4 per replica, 4 per lane with a ragged
# last pass) and 200 atoms (1200 floats = 300 float4, 10 per lane), with
# populations that end in a partly filled block.
@pytest.mark.parametrize("n,R", [(75, 1000), (75, 37), (200, 257), (200, 5)])
def test_gather_elementwise_large_molecules(lib, orc, n, R):
    top = pi.make_chain(n, 3)
    seed = 5 + R
    x = f32(pi.perturbed_positions(top, R, 0.05, 7))
    v = f32(pi.gaussian_velocities(R, n, 0.7, 8))
    E = pi.random_energies(R, -500.0, 40.0, 9)
    fam = (np.arange(R, dtype=np.int32) * 7 + 3) % 1009
    Tp, Tn = 800.0, 741.0
    ctx = lib.pamd_init(top, R, Tp, seed)
    try:
        lib.pamd_set_state(ctx, x, v, E, fam)
        cnt, lnq = lib.pamd_resample(ctx, Tp, Tn)
        xg, vg, eg, fg = lib.pamd_get_state(ctx)
    finally:
        lib.pamd_destroy(ctx)
    lnq_o, W = orc.resample_weights(E, Tp, Tn)
    cnt_o = orc.multinomial_counts(W, seed, 1)
    np.testing.assert_array_equal(cnt, cnt_o)
    xo, vo, fo, eo = orc.gather(top, cnt_o, x, v, fam, E, math.sqrt(Tn / Tp))
    np.testing.assert_array_equal(fg, fo)
    np.testing.assert_array_equal(eg, eo)
    # FP32 recentring (the centre of mass summed in FP32 per replica) and the
    # FP32 product with the velocity scale
    assert np.abs(xg - xo).max() < 4e-6 * max(1.0, np.abs(xo).max())
    assert np.abs(vg - vo).max() <= 2e-7 * np.abs(vo).max()


def test_consecutive_resamplings_bit_exact(lib, orc):
    """Every resampling of a sequence weighs the current population."""
    top = pi.make_chain(12, 3)
    R, seed, dt = 777, 5, 0.001
    temps = [900.0, 850.0, 800.0, 760.0, 720.0]
    ctx = lib.pamd_init(top, R, temps[0], seed)
    try:
        lib.pamd_propagate(ctx, 10, dt, temps[0])
        for i in range(1, len(temps)):
            _, _, E, _ = lib.pamd_get_state(ctx)
            cnt, lnq = lib.pamd_resample(ctx, temps[i - 1], temps[i])
            lnq_o, W = orc.resample_weights(E, temps[i - 1], temps[i])
            np.testing.assert_array_equal(cnt, orc.multinomial_counts(W, seed, i))
            assert abs(lnq - lnq_o) <= 1e-12 * max(1.0, abs(lnq_o))
            lib.pamd_propagate(ctx, 10, dt, temps[i])
    finally:
        lib.pamd_destroy(ctx)


def test_observables_match_oracle(lib, orc):
    top = pi.make_chain(22, 4)
    R = 3000
    ctx = lib.pamd_init(top, R, 600.0, 5)
    try:
        lib.pamd_propagate(ctx, 30, 0.001, 600.0)
        lib.pamd_resample(ctx, 600.0, 560.0)
        lib.pamd_propagate(ctx, 5, 0.001, 560.0)
        og = lib.pamd_observables(ctx, 560.0)
        x, v, E, fam = lib.pamd_get_state(ctx)
    finally:
        lib.pamd_destroy(ctx)
    oo = orc.observables(top, x, v, fam, E)
    for key in ("e_pot", "e_kin", "t_meas", "rg", "rg2"):
        assert abs(og[key] - oo[key]) <= 1e-9 * abs(oo[key]), key
    for key in ("e_pot_se", "e_kin_se", "rg_se", "rg2_se"):
        assert abs(og[key] - oo[key]) <= 1e-7 * abs(oo[key]) + 1e-12, key
    assert og["n_families"] == oo["n_families"]
    assert og["n_families"] < R  # resampling pruned some families


def test_anneal_graph_equals_stepwise_calls(lib):
    top = pi.make_chain(22, 1)
    temps = pi.geometric_schedule(1000.0, 600.0, 4)
    R, theta, dt = 256, 20, 0.001
    a = lib.pamd_init(top, R, temps[0], 3)
    b = lib.pamd_init(top, R, temps[0], 3)
    try:
        obs_a = lib.pamd_anneal(a, temps, theta, dt)
        obs_b = []
        lib.pamd_propagate(b, theta, dt, temps[0])
        obs_b.append(lib.pamd_observables(b, temps[0]))
        for i in range(1, len(temps)):
            lib.pamd_resample(b, temps[i - 1], temps[i], want_copies=False)
            lib.pamd_propagate(b, theta, dt, temps[i])
            obs_b.append(lib.pamd_observables(b, temps[i]))
        sa, sb = lib.pamd_get_state(a), lib.pamd_get_state(b)
        for u, w in zip(sa, sb):
            np.testing.assert_array_equal(u, w)
        for oa, ob in zip(obs_a, obs_b):
            for k in oa:
                assert oa[k] == ob[k], k
        assert lib.pamd_get_counters(a) == lib.pamd_get_counters(b)
        # a second graph launch continues with fresh counters
        obs_a2 = lib.pamd_anneal(a, temps, theta, dt)
        assert obs_a2[-1]["e_pot"] != obs_a[-1]["e_pot"]
    finally:
        lib.pamd_destroy(a)
        lib.pamd_destroy(b)


def test_c1_anneal_statistical_parity(lib, orc):
    """22-atom chain, R=256, theta=100, 20 geometric steps 1000 -> 300 K.

    Eight independent anneals (seeds) on each side.  One R = 256 anneal ends
    with a handful of families, so its family-binned error understates the
    spread of its means at low T and one realisation can sit 3 such errors
    away by chance; the run-to-run spread of eight runs is an honest error.
    The combined error of the two eight-run means takes, per side, the larger
    of the run-to-run standard error and the pooled family-binned error.
    """
    top = pi.make_chain(22, 1)
    temps = pi.geometric_schedule(1000.0, 300.0, 20)
    R, theta, dt, gamma = 256, 100, 0.001, 1.0
    seeds = [12345 + 1000 * k for k in range(8)]
    og, oo = [], []
    for sd in seeds:
        ctx = lib.pamd_init(top, R, temps[0], sd, _opts(lib, gamma_per_ps=gamma))
        try:
            og.append(lib.pamd_anneal(ctx, temps, theta, dt))
        finally:
            lib.pamd_destroy(ctx)
        oo.append(orc.anneal(top, R, temps, theta, dt, gamma, sd)[0])

    mean_and_se = _runs_mean_and_se

    # kinetic energy: theta = 100 is too short to equilibrate (the paper's
    # point about theta), so it is compared GPU against oracle, not against T
    for key, se in (("e_pot", "e_pot_se"), ("rg", "rg_se"), ("e_kin", "e_kin_se")):
        g, sg = mean_and_se(og, key, se)
        o, so = mean_and_se(oo, key, se)
        s = np.hypot(sg, so)
        assert np.all(np.abs(g - o) <= 3 * s), (key, (g - o) / s)


def test_c1_anneal_control_statistical_parity(lib, orc):
    """The resampling-off anneal (every copy kept once, velocities rescaled):
    same statistics as the oracle's, and no family is ever pruned."""
    top = pi.make_chain(22, 1)
    temps = pi.geometric_schedule(1000.0, 300.0, 20)
    R, theta, dt, gamma, seed = 256, 100, 0.001, 1.0, 4321
    ctx = lib.pamd_init(top, R, temps[0], seed, _opts(lib, gamma_per_ps=gamma))
    try:
        og = lib.pamd_anneal(ctx, temps, theta, dt, resample=False)
        _, _, _, fam = lib.pamd_get_state(ctx)
    finally:
        lib.pamd_destroy(ctx)
    oo, _, _, ofam, _ = orc.anneal(top, R, temps, theta, dt, gamma, seed, resample=False)
    np.testing.assert_array_equal(fam, np.arange(R))
    np.testing.assert_array_equal(ofam, np.arange(R))
    assert all(o["n_families"] == R for o in og)
    for key, se in (("e_pot", "e_pot_se"), ("e_kin", "e_kin_se"), ("rg", "rg_se")):
        g = np.array([o[key] for o in og])
        o = np.array([o[key] for o in oo])
        s = np.sqrt(np.array([x[se] for x in og]) ** 2 + np.array([x[se] for x in oo]) ** 2)
        assert np.all(np.abs(g - o) <= 3 * s), (key, (g - o) / s)
    # ln Q is still recorded (it estimates the free-energy steps from the
    # unresampled population); the two sides agree statistically
    lg = np.array([o["sum_lnQ"] for o in og]); lo = np.array([o["sum_lnQ"] for o in oo])
    assert np.all(np.abs(lg - lo) <= 0.05 * np.abs(lo) + 1.0), lg - lo


def test_harmonic_chain_closed_forms_on_gpu(lib):
    """Bonds-only chain (r0 = 0): <E_pot>(T) = (3/2)(N-1) k_B T and
    sum ln Q = (3/2)(N-1) ln(T/T0) at every temperature.  BAOAB samples the
    configurations of a harmonic potential exactly at any stable step size
    (Leimkuhler & Matthews 2013), and resampling plus velocity rescaling carry
    the population to each new temperature exactly up to the finite-population
    bias, so no step-size allowance is needed.  The population is first
    equilibrated at T0 for 4 ps (20 friction times; the anneal's own first
    block is 0.4 ps, half a bond period).  Eight independent anneals, the
    mean within 3 standard errors (run-to-run or pooled family-binned, the
    larger) of the closed form."""
    n, kb = 6, 400.0
    top = pi.make_harmonic_chain(n, kb, 0.0)
    temps = pi.geometric_schedule(400.0, 200.0, 6)
    runs = []
    for k in range(8):
        ctx = lib.pamd_init(top, 4096, temps[0], 11 + 7 * k, _opts(lib, gamma_per_ps=5.0))
        try:
            lib.pamd_propagate(ctx, 2000, 0.002, temps[0])
            runs.append(lib.pamd_anneal(ctx, temps, 200, 0.002))
        finally:
            lib.pamd_destroy(ctx)
    e, se = _runs_mean_and_se(runs, "e_pot", "e_pot_se")
    e_exact = 1.5 * (n - 1) * KB * temps
    assert np.all(np.abs(e - e_exact) <= 3 * se), (e - e_exact) / se
    f = np.array([[o["sum_lnQ"] for o in r] for r in runs])
    f_exact = 1.5 * (n - 1) * np.log(temps / temps[0])
    f_se = np.maximum(f.std(0, ddof=1) / np.sqrt(len(runs)), 1e-12)
    assert np.all(np.abs(f.mean(0) - f_exact) <= 3 * f_se + 1e-9), (f.mean(0) - f_exact) / f_se


def test_nonfinite_energy_is_reported(lib):
    top = pi.make_chain(6, 1)
    R = 4
    x = f32(pi.perturbed_positions(top, R, 0.01, 1))
    x[2, 5] = x[2, 0]  # a non-excluded pair on top of each other
    ctx = lib.pamd_init(top, R, 300.0, 1)
    try:
        lib.pamd_set_state(ctx, x, np.zeros_like(x))
        with pytest.raises(lib.PamdError) as ei:
            lib.pamd_forces(ctx)
        assert ei.value.code == lib.PAMD_ENONFINITE and "replica 2" in str(ei.value)
        # the context stays usable once the state is repaired
        x[2, 5] = x[1, 5]
        lib.pamd_set_state(ctx, x, np.zeros_like(x))
        f, E = lib.pamd_forces(ctx)
        assert np.all(np.isfinite(E))
    finally:
        lib.pamd_destroy(ctx)


def test_checkpoint_resume_is_bit_identical(lib):
    top = pi.make_chain(22, 2)
    R, dt = 300, 0.001
    a = lib.pamd_init(top, R, 900.0, 21)
    b = lib.pamd_init(top, R, 900.0, 21)
    c = lib.pamd_init(top, R, 900.0, 21)
    try:
        for ctx in (a, b):
            lib.pamd_propagate(ctx, 25, dt, 900.0)
        lib.pamd_resample(a, 900.0, 850.0)
        lib.pamd_propagate(a, 25, dt, 850.0)
        # checkpoint b, restore into c, continue there
        x, v, E, fam = lib.pamd_get_state(b)
        ctr = lib.pamd_get_counters(b)
        lib.pamd_set_state(c, x, v, E, fam)
        lib.pamd_set_counters(c, *ctr)
        lib.pamd_resample(c, 900.0, 850.0)
        lib.pamd_propagate(c, 25, dt, 850.0)
        for u, w in zip(lib.pamd_get_state(a), lib.pamd_get_state(c)):
            np.testing.assert_array_equal(u, w)
        assert lib.pamd_get_counters(a) == lib.pamd_get_counters(c)
    finally:
        for ctx in (a, b, c):
            lib.pamd_destroy(ctx)


def test_torch_allocator_and_stream(lib):
    import torch
    top = pi.make_chain(22, 5)
    temps = pi.geometric_schedule(800.0, 700.0, 2)
    a = lib.Population(top, 128, temps[0], 8, lib.torch_options())
    b = lib.Population(top, 128, temps[0], 8)
    try:
        before = torch.cuda.memory_allocated()
        assert before > 0  # the population lives in PyTorch's allocator
        oa = a.anneal(temps, 10, 0.001)
        ob = b.anneal(temps, 10, 0.001)
        assert oa == ob
    finally:
        a.close()
        b.close()


def test_full_size_sampled_parity(lib, orc):
    """75-atom chain, R = 8192 (the benchmark shape): the full launch, checked on
    sampled replicas against the oracle, and the full-size resampling bit-exact."""
    top = pi.make_chain(75, 1)
    R, T, dt, seed = 8192, 1000.0, 0.001, 12345
    ctx = lib.pamd_init(top, R, T, seed)
    try:
        x0, v0, _, _ = lib.pamd_get_state(ctx)
        lib.pamd_propagate(ctx, 10, dt, T)
        x1, v1, E1, fam = lib.pamd_get_state(ctx)
        cnt, lnq = lib.pamd_resample(ctx, T, 980.0)
    finally:
        lib.pamd_destroy(ctx)
    sample = np.array([0, 1, 31, 32, 33, 1000, 4095, 4096, 8190, 8191])
    xo, vo, eo = orc.propagate(top, x0[sample], v0[sample], 10, dt, T, 1.0, seed, 0, slots=sample)
    assert np.abs(x1[sample] - xo).max() < 1e-4
    assert np.abs(E1[sample] - eo).max() < 1e-4 * np.abs(eo).max()
    lnq_o, W = orc.resample_weights(E1, T, 980.0)
    np.testing.assert_array_equal(cnt, orc.multinomial_counts(W, seed, 1))
    assert abs(lnq - lnq_o) <= 1e-12 * max(1.0, abs(lnq_o))


def test_large_population_resample_bit_exact(lib, orc):
    """R = 2^20 replicas of the 75-atom chain: copy counts bit-exact."""
    top = pi.make_chain(75, 1)
    R, seed = 1 << 20, 31
    ctx = lib.pamd_init(top, R, 1000.0, seed)
    try:
        lib.pamd_propagate(ctx, 2, 0.001, 1000.0)
        _, _, E, _ = lib.pamd_get_state(ctx, positions=False, velocities=False, families=False)
        cnt, lnq = lib.pamd_resample(ctx, 1000.0, 975.0)
    finally:
        lib.pamd_destroy(ctx)
    lnq_o, W = orc.resample_weights(E, 1000.0, 975.0)
    np.testing.assert_array_equal(cnt, orc.multinomial_counts(W, seed, 1))
    assert abs(lnq - lnq_o) <= 1e-11 * max(1.0, abs(lnq_o))


def test_autotune_keeps_state_and_parity(lib, orc):
    top = pi.make_chain(75, 1)
    R = 600
    ctx = lib.pamd_init(top, R, 800.0, 3)
    try:
        lib.pamd_propagate(ctx, 5, 0.001, 800.0)
        before = lib.pamd_get_state(ctx)
        ctr = lib.pamd_get_counters(ctx)
        tune = lib.pamd_autotune(ctx, 5)
        assert tune["from_cache"] == 0 and tune["ms"] > 0
        assert tune["lanes_per_replica"] * tune["atoms_per_lane"] >= 75
        for u, w in zip(before, lib.pamd_get_state(ctx)):
            np.testing.assert_array_equal(u, w)
        assert lib.pamd_get_counters(ctx) == ctr
        info = lib.pamd_info(ctx)
        assert info["lanes_per_replica"] == tune["lanes_per_replica"]
        # the tuned shape computes the same forces
        x = before[0][:4]
        fg, eg = lib.pamd_forces(ctx)
        fo, eo, scale = _oracle_forces(orc, top, before[0][:4])
        for k in range(4):
            rms = math.sqrt(np.mean(fo[k] ** 2))
            assert math.sqrt(np.mean((fg[k] - fo[k]) ** 2)) <= 1e-5 * rms
        assert lib.pamd_autotune(ctx, 5)["from_cache"] == 1
    finally:
        lib.pamd_destroy(ctx)


def test_checkpoint_file_roundtrip(lib, tmp_path):
    """A run restored from a checkpoint file continues bit-identically;
    corrupt or foreign files are refused and leave the population unchanged."""
    top = pi.make_chain(22, 5)
    temps = pi.geometric_schedule(900.0, 700.0, 2)
    path = str(tmp_path / "run.ckpt")
    pop = lib.Population(top, 300, temps[0], 21)
    other = lib.Population(top, 301, temps[0], 21)
    try:
        pop.propagate(15, 0.001, temps[0])
        pop.resample(temps[0], temps[1], want_copies=False)
        pop.checkpoint(path)
        pop.propagate(15, 0.001, temps[1])
        pop.resample(temps[1], temps[2], want_copies=False)
        a = pop.state()
        ca = lib.pamd_get_counters(pop.ctx)
        pop.reset(temps[0], 99)            # scramble, then come back
        pop.propagate(3, 0.001, temps[0])
        pop.restore(path)
        pop.propagate(15, 0.001, temps[1])
        pop.resample(temps[1], temps[2], want_copies=False)
        b = pop.state()
        for u, w in zip(a, b):
            np.testing.assert_array_equal(u, w)
        assert lib.pamd_get_counters(pop.ctx) == ca
        # corrupt: flip one payload byte
        raw = bytearray(open(path, "rb").read())
        raw[200] ^= 0x40
        bad = str(tmp_path / "bad.ckpt")
        open(bad, "wb").write(bytes(raw))
        before = pop.state()
        with pytest.raises(lib.PamdError) as e:
            pop.restore(bad)
        assert e.value.code == lib.PAMD_EINVAL
        for u, w in zip(before, pop.state()):
            np.testing.assert_array_equal(u, w)
        with pytest.raises(lib.PamdError):
            other.restore(path)            # another population size
    finally:
        pop.close()
        other.close()


def test_75_atom_anneal_statistical_parity(lib, orc):
    """The benchmark's 75-atom chain: R = 512, theta = 200, 20 geometric
    steps 1000 -> 250 K, eight independent anneals on each side; <E_pot>(T)
    and <R_g>(T) within 3 combined standard errors of the oracle, for the
    scalar and for the packed pair arithmetic (whichever the tuner picks runs
    the benchmark)."""
    top = pi.make_chain(75, 1)
    temps = pi.geometric_schedule(1000.0, 250.0, 20)
    R, theta, dt, gamma = 512, 200, 0.001, 1.0
    seeds = [777 + 1000 * k for k in range(8)]
    oo = [orc.anneal(top, R, temps, theta, dt, gamma, sd)[0] for sd in seeds]
    for arith in (lib.PAMD_PAIRS_SCALAR, lib.PAMD_PAIRS_PACKED):
        og = []
        for sd in seeds:
            ctx = lib.pamd_init(top, R, temps[0], sd + 1, _opts(lib, gamma_per_ps=gamma,
                                                               pair_arith=arith))
            try:
                og.append(lib.pamd_anneal(ctx, temps, theta, dt))
            finally:
                lib.pamd_destroy(ctx)
        for key, se in (("e_pot", "e_pot_se"), ("rg", "rg_se")):
            g, sg = _runs_mean_and_se(og, key, se)
            o, so = _runs_mean_and_se(oo, key, se)
            s = np.hypot(sg, so)
            assert np.all(np.abs(g - o) <= 3 * s), (arith, key, (g - o) / s)


def test_batched_anneal_statistical_parity(lib, orc):
    """Three molecules of uneven size annealed by one batch context (one
    persistent launch per temperature block) against the oracle run on each
    molecule alone: per molecule, <E_pot>(T) and <R_g>(T) over eight seeds
    within 3 combined standard errors."""
    sizes = [20, 31, 47]
    tops = [pi.make_chain(n, 40 + n) for n in sizes]
    temps = pi.geometric_schedule(800.0, 300.0, 10)
    R, theta, dt, gamma = 256, 100, 0.001, 1.0
    seeds = [31 + 97 * k for k in range(8)]
    gb = [[] for _ in sizes]
    for sd in seeds:
        ctx = lib.pamd_init_batch(tops, [R] * len(sizes), [temps[0]] * len(sizes), sd,
                                  _opts(lib, gamma_per_ps=gamma))
        try:
            obs = lib.pamd_anneal(ctx, temps, theta, dt)
        finally:
            lib.pamd_destroy(ctx)
        for m in range(len(sizes)):
            gb[m].append([row[m] for row in obs])
    for m, top in enumerate(tops):
        oo = [orc.anneal(top, R, temps, theta, dt, gamma, sd + 5, mol=m)[0] for sd in seeds]
        for key, se in (("e_pot", "e_pot_se"), ("rg", "rg_se")):
            g, sg = _runs_mean_and_se(gb[m], key, se)
            o, so = _runs_mean_and_se(oo, key, se)
            s = np.hypot(sg, so)
            assert np.all(np.abs(g - o) <= 3 * s), (sizes[m], key, (g - o) / s)
