"""Batched uneven anneals: many molecules in one persistent launch.

* Every molecule of a batch advances exactly as a standalone context with the
  same launch shape, pair arithmetic and molecule index would (same kernel
  body, same Philox stream), and matches the FP64 oracle over 10 steps;
  chains take the packed pair arithmetic unless the scalar one is asked for.
* Resampling, observables and the graph-captured anneal act per molecule.
* The 16-molecule workload (N ~ U{20..200}, 4096 replicas each) runs and
  sampled replicas match the oracle.
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


def _sub_opts(lib, sub):
    info = lib.pamd_info(sub)
    o = lib.pamd_options_default()
    o.lanes_per_replica = info["lanes_per_replica"]
    o.warps_per_block = 4
    o.pair_arith = lib.pamd_get_shape(sub)["pair_arith"]
    return o


def test_batch_matches_standalone_and_oracle(lib, orc):
    sizes, Rs = [22, 75, 45], [300, 257, 128]
    tops = [pi.make_chain(n, 10 + n) for n in sizes]
    T, dt, seed = 600.0, 0.001, 77
    batch = lib.pamd_init_batch(tops, Rs, [T] * 3, seed)
    try:
        assert lib.pamd_batch_size(batch) == 3
        subs = [lib.pamd_batch_sub(batch, m) for m in range(3)]
        # chains take the packed pair arithmetic in a batch
        assert all(lib.pamd_get_shape(s_)["pair_arith"] == lib.PAMD_PAIRS_PACKED for s_ in subs)
        starts = [lib.pamd_get_state(s) for s in subs]
        lib.pamd_propagate(batch, 10, dt, T)
        for m, (top, R, sub) in enumerate(zip(tops, Rs, subs)):
            xb, vb, Eb, _ = lib.pamd_get_state(sub)
            # standalone context: same shape, same molecule index, same start
            o = _sub_opts(lib, sub)
            o.mol_id = m
            ctx = lib.pamd_init(top, R, T, seed, o)
            try:
                lib.pamd_set_state(ctx, starts[m][0], starts[m][1])
                lib.pamd_propagate(ctx, 10, dt, T)
                xs, vs, Es, _ = lib.pamd_get_state(ctx)
            finally:
                lib.pamd_destroy(ctx)
            assert np.abs(xb - xs).max() < 1e-5
            np.testing.assert_allclose(Eb, Es, rtol=1e-5, atol=1e-4)
            # oracle, sampled replicas, same molecule stream
            sample = np.array([0, R // 2, R - 1])
            xo, vo, eo = orc.propagate(top, starts[m][0][sample], starts[m][1][sample], 10, dt, T,
                                       1.0, seed, 0, mol=m, slots=sample)
            assert np.abs(xb[sample] - xo).max() < 1e-4
    finally:
        lib.pamd_destroy(batch)


def test_batch_resample_observables_and_anneal(lib, orc):
    sizes, Rs = [30, 60], [512, 300]
    tops = [pi.make_chain(n, 3 + n) for n in sizes]
    temps = pi.geometric_schedule(900.0, 700.0, 3)
    seed = 5
    batch = lib.pamd_init_batch(tops, Rs, [temps[0]] * 2, seed)
    try:
        subs = [lib.pamd_batch_sub(batch, m) for m in range(2)]
        lib.pamd_propagate(batch, 20, 0.001, temps[0])
        E = [lib.pamd_get_state(s)[2] for s in subs]
        cnt, lnq = lib.pamd_resample(batch, temps[0], temps[1])
        assert len(lnq) == 2 and cnt.shape == (sum(Rs),)
        off = 0
        for m in range(2):
            lnq_o, W = orc.resample_weights(E[m], temps[0], temps[1])
            np.testing.assert_array_equal(cnt[off:off + Rs[m]],
                                          orc.multinomial_counts(W, seed, 1, mol=m))
            assert abs(lnq[m] - lnq_o) < 1e-12 * max(1.0, abs(lnq_o))
            off += Rs[m]
        obs = lib.pamd_observables(batch, temps[1])
        assert len(obs) == 2 and all(o["n_families"] <= R for o, R in zip(obs, Rs))
        # graph-captured anneal of the whole batch, twice (fresh counters)
        lib.pamd_reset(batch, temps[0], seed)
        a = lib.pamd_anneal(batch, temps, 15, 0.001)
        assert len(a) == len(temps) and len(a[0]) == 2
        assert all(math.isfinite(a[i][m]["e_pot"]) for i in range(len(temps)) for m in range(2))
        b = lib.pamd_anneal(batch, temps, 15, 0.001)
        assert b[-1][0]["e_pot"] != a[-1][0]["e_pot"]
    finally:
        lib.pamd_destroy(batch)


def test_batch_anneal_matches_stepwise(lib):
    tops = [pi.make_chain(n, n) for n in (25, 50)]
    temps = pi.geometric_schedule(800.0, 650.0, 2)
    A = lib.pamd_init_batch(tops, [200, 150], [temps[0]] * 2, 9)
    B = lib.pamd_init_batch(tops, [200, 150], [temps[0]] * 2, 9)
    try:
        ga = lib.pamd_anneal(A, temps, 10, 0.001)
        lib.pamd_propagate(B, 10, 0.001, temps[0])
        gb = [lib.pamd_observables(B, temps[0])]
        for i in range(1, len(temps)):
            lib.pamd_resample(B, temps[i - 1], temps[i], want_copies=False)
            lib.pamd_propagate(B, 10, 0.001, temps[i])
            gb.append(lib.pamd_observables(B, temps[i]))
        for ra, rb in zip(ga, gb):
            for oa, ob in zip(ra, rb):
                assert oa == ob
        for m in range(2):
            for u, w in zip(lib.pamd_get_state(lib.pamd_batch_sub(A, m)),
                            lib.pamd_get_state(lib.pamd_batch_sub(B, m))):
                np.testing.assert_array_equal(u, w)
    finally:
        lib.pamd_destroy(A)
        lib.pamd_destroy(B)


def test_batch_scalar_arithmetic_on_request(lib, orc):
    """pair_arith = PAMD_PAIRS_SCALAR keeps every molecule of a batch on the
    scalar pair arithmetic, and that batch matches the oracle as well."""
    sizes, R = [22, 75], 128
    tops = [pi.make_chain(n, 40 + n) for n in sizes]
    T, dt, seed = 650.0, 0.001, 19
    o = lib.pamd_options_default()
    o.pair_arith = lib.PAMD_PAIRS_SCALAR
    batch = lib.pamd_init_batch(tops, [R] * 2, [T] * 2, seed, o)
    try:
        subs = [lib.pamd_batch_sub(batch, m) for m in range(2)]
        assert all(lib.pamd_get_shape(s_)["pair_arith"] == lib.PAMD_PAIRS_SCALAR for s_ in subs)
        starts = [lib.pamd_get_state(s_) for s_ in subs]
        lib.pamd_propagate(batch, 8, dt, T)
        for m in range(2):
            x, _, _, _ = lib.pamd_get_state(subs[m])
            sample = np.array([0, R - 1])
            xo, _, _ = orc.propagate(tops[m], starts[m][0][sample], starts[m][1][sample], 8, dt, T,
                                     1.0, seed, 0, mol=m, slots=sample)
            assert np.abs(x[sample] - xo).max() < 1e-4
    finally:
        lib.pamd_destroy(batch)


def test_batch_chain_with_far_exclusions(lib, orc):
    """A batch holding a standard chain and a chain with extra exclusions
    between distant atoms (masked pairs beyond the first ring step): both run
    the packed batched kernel and match the oracle."""
    sizes, R = [40, 75], 96
    tops = [pi.make_chain(n, 50 + n) for n in sizes]
    far = [(2, 37), (10, 70), (0, 74), (5, 50)]
    tops[1].excl = np.concatenate([np.asarray(tops[1].excl, np.int32).reshape(-1, 2),
                                   np.asarray(far, np.int32)]).astype(np.int32)
    T, dt, seed = 550.0, 0.001, 23
    batch = lib.pamd_init_batch(tops, [R] * 2, [T] * 2, seed)
    try:
        subs = [lib.pamd_batch_sub(batch, m) for m in range(2)]
        assert all(lib.pamd_get_shape(s_)["pair_arith"] == lib.PAMD_PAIRS_PACKED for s_ in subs)
        starts = [lib.pamd_get_state(s_) for s_ in subs]
        lib.pamd_propagate(batch, 8, dt, T)
        for m in range(2):
            x, _, E, _ = lib.pamd_get_state(subs[m])
            sample = np.array([0, R // 3, R - 1])
            xo, _, eo = orc.propagate(tops[m], starts[m][0][sample], starts[m][1][sample], 8, dt, T,
                                      1.0, seed, 0, mol=m, slots=sample)
            assert np.abs(x[sample] - xo).max() < 1e-4
            assert np.abs(E[sample] - eo).max() < 1e-4 * np.abs(eo).max()
    finally:
        lib.pamd_destroy(batch)


def test_sixteen_uneven_molecules(lib, orc):
    """The batched workload shape: 16 chains, N ~ U{20..200}, 4096 replicas each."""
    sizes = pi.batched_chain_sizes()
    tops = [pi.make_chain(n, m + 1) for m, n in enumerate(sizes)]
    R, T, dt, seed = 4096, 800.0, 0.001, 12345
    batch = lib.pamd_init_batch(tops, [R] * 16, [T] * 16, seed)
    try:
        subs = [lib.pamd_batch_sub(batch, m) for m in range(16)]
        pick = [int(np.argmin(sizes)), int(np.argmax(sizes)), 7]
        starts = {m: lib.pamd_get_state(subs[m]) for m in pick}
        lib.pamd_propagate(batch, 5, dt, T)
        for m in pick:
            x, _, E, _ = lib.pamd_get_state(subs[m])
            sample = np.array([0, 2049, R - 1])
            xo, vo, eo = orc.propagate(tops[m], starts[m][0][sample], starts[m][1][sample], 5, dt, T,
                                       1.0, seed, 0, mol=m, slots=sample)
            assert np.abs(x[sample] - xo).max() < 1e-4
            assert np.abs(E[sample] - eo).max() < 1e-4 * np.abs(eo).max()
    finally:
        lib.pamd_destroy(batch)


def test_batch_autotuned_shapes(lib, orc):
    """With autotuning each molecule gets a measured shape among the batched
    kernel's (3..7 atoms per lane), and the batch still matches the oracle."""
    sizes, R = [22, 75, 130], 256
    tops = [pi.make_chain(n, 30 + n) for n in sizes]
    T, dt, seed = 700.0, 0.001, 5
    o = lib.pamd_options_default()
    o.autotune = 1
    batch = lib.pamd_init_batch(tops, [R] * 3, [T] * 3, seed, o)
    try:
        subs = [lib.pamd_batch_sub(batch, m) for m in range(3)]
        for s_ in subs:
            assert 3 <= lib.pamd_info(s_)["atoms_per_lane"] <= 7
        starts = [lib.pamd_get_state(s_) for s_ in subs]
        lib.pamd_propagate(batch, 6, dt, T)
        for m in range(3):
            x, _, _, _ = lib.pamd_get_state(subs[m])
            sample = np.array([0, R - 1])
            xo, _, _ = orc.propagate(tops[m], starts[m][0][sample], starts[m][1][sample], 6, dt, T,
                                     1.0, seed, 0, mol=m, slots=sample)
            assert np.abs(x[sample] - xo).max() < 1e-4
    finally:
        lib.pamd_destroy(batch)
