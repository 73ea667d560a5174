"""The learned surrogate on the GPU, held to the FP64 oracle (oracle/mlp.py).

* The tensor-core GEMM is exact on small-integer BF16 operands (every
  product and partial sum is an integer below 2^24) and within the FP32
  accumulation bound K 2^-22 sum |a||b| on Gaussian operands, over shapes
  with ragged M, N and K tails.
* Energies and forces match the oracle evaluated with the same BF16-rounded
  weights; the remaining difference is the BF16 rounding of features and
  activations (tolerance 2e-2 relative, see below).
* The training gradient of the force-matching loss matches the oracle on a
  small batch; Adam on GPU-harvested exact data lowers the force error.
* The torch.autograd.Function's backward (the force kernel) agrees with the
  slope of its own forward along random directions.
* Surrogate-driven BAOAB trajectories match the oracle integrator.

Tolerances: BF16 keeps 8 significant bits, so each rounding of a normalised
feature, hidden activation or back-propagated signal has relative error at
most 2^-9 ~ 2e-3.  Errors of the ~10^2..10^3 independently rounded terms of
a dot product add in quadrature and are damped by the fan-in normalisation;
the end-to-end relative error of E (in units of sigma_E) and of the force
RMS is therefore a few 1e-3.  The tests use 2e-2 (energy, forces) and 3e-2
(gradients, which pass through two more BF16 roundings).
"""
import numpy as np
import pytest

import pamd_inputs as pi
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_06016_gb300 import build, pamd, surrogate
    build.build()
    pamd.load()
    return torch, pamd, surrogate


def bf16_round(a):
    """Round float32 values to the nearest BF16 (ties to even), returned as float64."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def _bf16_tensor(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda().to(torch.bfloat16)


GEMM_SHAPES = [(128, 128, 64), (1, 1, 8), (200, 300, 72), (129, 257, 136), (1000, 512, 2776),
               (512, 2776, 512), (512, 512, 8), (384, 640, 520)]


@pytest.mark.parametrize("M,N,K", GEMM_SHAPES)
def test_gemm_exact_on_small_integers(env, M, N, K):
    torch, _, S = env
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.integers(-4, 5, (M, K)).astype(np.float64)
    B = rng.integers(-4, 5, (N, K)).astype(np.float64)
    C = S.gemm_bf16(_bf16_tensor(torch, A), _bf16_tensor(torch, B)).cpu().numpy()
    np.testing.assert_array_equal(C, A @ B.T)


@pytest.mark.parametrize("M,N,K", GEMM_SHAPES)
def test_gemm_within_fp32_accumulation_bound(env, M, N, K):
    torch, _, S = env
    rng = np.random.default_rng(M + 11 * N + 13 * K)
    A = bf16_round(rng.normal(0, 1, (M, K)))
    B = bf16_round(rng.normal(0, 1, (N, K)))
    C = S.gemm_bf16(_bf16_tensor(torch, A), _bf16_tensor(torch, B)).cpu().numpy()
    bound = K * 2.0 ** -22 * (np.abs(A) @ np.abs(B).T)
    assert np.all(np.abs(C - A @ B.T) <= bound)


# Shapes of the surrogate's production calls: far more 128 x 256 tile pairs
# than the 76 resident two-CTA clusters, so every cluster walks several tiles,
# both tensor-memory accumulators are used and the TMA ring wraps across tiles.
FULL_SIZE_SHAPES = [(40000, 512, 2776), (65536, 512, 512)]


@pytest.mark.parametrize("M,N,K", FULL_SIZE_SHAPES)
def test_gemm_full_size_multi_tile(env, M, N, K):
    torch, _, S = env
    rng = np.random.default_rng(M + N + K)
    # small integers: every partial sum is an integer below 2^24, so the
    # product is exact and a float32 product on the host is exact as well
    A = rng.integers(-4, 5, (M, K)).astype(np.float32)
    B = rng.integers(-4, 5, (N, K)).astype(np.float32)
    C = S.gemm_bf16(_bf16_tensor(torch, A), _bf16_tensor(torch, B)).cpu().numpy()
    np.testing.assert_array_equal(C, A @ B.T)
    # Gaussian operands within the FP32 accumulation bound, on sampled rows of
    # every cluster's tiles (rows from all 128-row blocks)
    A = bf16_round(rng.normal(0, 1, (M, K))).astype(np.float32)
    B = bf16_round(rng.normal(0, 1, (N, K))).astype(np.float32)
    C = S.gemm_bf16(_bf16_tensor(torch, A), _bf16_tensor(torch, B)).cpu().numpy()
    rows = np.unique(np.concatenate([np.arange(0, M, 97), [M - 1]]))
    A64, B64 = A[rows].astype(np.float64), B.astype(np.float64)
    bound = K * 2.0 ** -22 * (np.abs(A64) @ np.abs(B64).T)
    assert np.all(np.abs(C[rows] - A64 @ B64.T) <= bound)


def test_gemm_rejects_memory_of_another_device(env):
    """The B tile is multicast by TMA into both CTAs of a cluster, so the
    operands must be device memory of the current GPU: host memory and
    page-locked host memory (torch's pin_memory, a cudaHostAlloc allocation
    with the default flags, i.e. what cudaMallocHost returns) are refused."""
    torch, pamd, _ = env
    lib = pamd.load()
    M = N = K = 64
    dev = torch.ones((M, K), dtype=torch.bfloat16, device="cuda")
    out = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    raw = np.zeros(M * K + 64, np.uint16)
    off = (-raw.ctypes.data % 64) // 2
    host = raw[off:off + M * K]
    pinned = torch.ones((M, K), dtype=torch.bfloat16).pin_memory()
    for bad in (host.ctypes.data, pinned.data_ptr()):
        assert lib.pamd_gemm_bf16(bad, dev.data_ptr(), out.data_ptr(), M, N, K, K, K, N, None) \
            == pamd.PAMD_EINVAL
        assert lib.pamd_gemm_bf16(dev.data_ptr(), bad, out.data_ptr(), M, N, K, K, K, N, None) \
            == pamd.PAMD_EINVAL
    # device operands still work afterwards
    assert lib.pamd_gemm_bf16(dev.data_ptr(), dev.data_ptr(), out.data_ptr(), M, N, K, K, K, N,
                              None) == 0
    torch.cuda.synchronize()
    assert torch.all(out == K)


def _model_and_params(env, n, hidden, seed, x):
    """A GPU model with non-trivial normalisation and biases, and the oracle's
    FP64 copy of it with the BF16-rounded weights the tensor cores use."""
    torch, _, S = env
    model = S.MLP(n, hidden, seed=seed)
    p = model.get_params()
    rng = np.random.default_rng(seed + 100)
    g = omlp.features(x)
    p["mu"] = g.mean(0).astype(np.float32)
    p["sd"] = (g.std(0) + 0.05).astype(np.float32)
    p["b1"] = rng.normal(0, 0.3, hidden).astype(np.float32)
    p["b2"] = rng.normal(0, 0.3, hidden).astype(np.float32)
    p["b3"], p["mu_E"], p["sigma_E"] = 0.25, -40.0, 15.0
    model.set_params(p)
    q = {k: (np.asarray(v, dtype=np.float64) if isinstance(v, np.ndarray) else float(v))
         for k, v in model.get_params().items()}
    q["W1"] = bf16_round(q["W1"])
    q["W2"] = bf16_round(q["W2"])
    return model, q


@pytest.mark.parametrize("n,hidden,M", [(22, 128, 64), (75, 512, 48), (9, 64, 300), (150, 64, 16)])
def test_energy_forces_match_oracle(env, n, hidden, M):
    torch, _, _ = env
    x = pi.perturbed_positions(pi.make_chain(n, n), M, 0.03, 1)
    model, q = _model_and_params(env, n, hidden, n + hidden, x)
    try:
        E, F = model.energy_forces(torch.from_numpy(x.astype(np.float32)).cuda())
        E, F = E.cpu().numpy(), F.cpu().numpy()
        Eo, Fo = omlp.energy_forces(q, x.astype(np.float32).astype(np.float64))
        assert np.abs(E - Eo).max() <= 2e-2 * q["sigma_E"]
        assert np.sqrt(np.mean((F - Fo) ** 2)) <= 2e-2 * np.sqrt(np.mean(Fo ** 2))
        # energy without the backward pass is the same number
        E2, _ = model.energy_forces(torch.from_numpy(x.astype(np.float32)).cuda(), forces=False)
        np.testing.assert_array_equal(E2.cpu().numpy(), E)
    finally:
        model.close()


def test_energy_forces_full_size_sampled(env):
    """75 atoms, 20 000 configurations: the GEMMs run the persistent
    multi-tile path of production calls; 64 sampled rows against the oracle."""
    torch, _, _ = env
    n, hidden, M = 75, 512, 20000
    top = pi.make_chain(n, 1)
    x = pi.perturbed_positions(top, M, 0.03, 11)
    model, q = _model_and_params(env, n, hidden, 77, x[:2000])
    try:
        E, F = model.energy_forces(torch.from_numpy(x.astype(np.float32)).cuda())
        E, F = E.cpu().numpy(), F.cpu().numpy()
        rows = np.unique(np.linspace(0, M - 1, 64).astype(int))
        assert len(rows) >= 64
        Eo, Fo = omlp.energy_forces(q, x[rows].astype(np.float32).astype(np.float64))
        assert np.abs(E[rows] - Eo).max() <= 2e-2 * q["sigma_E"]
        assert np.sqrt(np.mean((F[rows] - Fo) ** 2)) <= 2e-2 * np.sqrt(np.mean(Fo ** 2))
    finally:
        model.close()


@pytest.mark.parametrize("lam", [0.0, 0.8])
def test_loss_gradient_matches_oracle(env, lam):
    torch, _, _ = env
    n, hidden, M = 22, 128, 8
    x = pi.perturbed_positions(pi.make_chain(n, 4), M, 0.03, 2).astype(np.float32)
    model, q = _model_and_params(env, n, hidden, 7, x.astype(np.float64))
    rng = np.random.default_rng(5)
    E_ref = -40.0 + 15.0 * rng.normal(0, 1, M)
    F_ref = rng.normal(0, 200.0, (M, n, 3)).astype(np.float32)
    try:
        xt = torch.from_numpy(x).cuda()
        L = model.loss_grads(xt, torch.from_numpy(E_ref).cuda(), torch.from_numpy(F_ref).cuda(),
                             lam=lam)
        g = model.get_grads()
        Lo, go = omlp.loss_and_grads(q, x.astype(np.float64), E_ref, F_ref.astype(np.float64), lam)
        assert abs(L - Lo) <= 3e-2 * abs(Lo)
        for k in ("W1", "b1", "W2", "b2", "w3"):
            err = np.linalg.norm(g[k] - go[k]) / np.linalg.norm(go[k])
            assert err <= 3e-2, (k, err)
        assert abs(g["b3"] - go["b3"]) <= 3e-2 * abs(go["b3"]) + 1e-6
        # a minibatch selected by index gives the gradient of those samples
        idx = torch.tensor([6, 1, 3, 0], dtype=torch.int32, device="cuda")
        model.loss_grads(xt, torch.from_numpy(E_ref).cuda(), torch.from_numpy(F_ref).cuda(),
                         idx=idx, lam=lam)
        gi = model.get_grads()
        sel = [6, 1, 3, 0]
        _, gs = omlp.loss_and_grads(q, x[sel].astype(np.float64), E_ref[sel],
                                    F_ref[sel].astype(np.float64), lam)
        assert np.linalg.norm(gi["W1"] - gs["W1"]) <= 3e-2 * np.linalg.norm(gs["W1"])
    finally:
        model.close()


def test_autograd_backward_matches_slope_of_forward(env):
    torch, _, S = env
    n, M = 22, 6
    x = pi.perturbed_positions(pi.make_chain(n, 8), M, 0.03, 3)
    model, _ = _model_and_params(env, n, 128, 9, x)
    try:
        xt = torch.from_numpy(x.astype(np.float32)).cuda().requires_grad_(True)
        E = S.surrogate_energy(xt, model)
        w = torch.linspace(0.5, 1.5, M, device="cuda", dtype=torch.float64)
        (E * w).sum().backward()
        grad = xt.grad.double().cpu().numpy()
        rng = np.random.default_rng(4)
        v = rng.normal(0, 1, x.shape)
        v /= np.linalg.norm(v.reshape(M, -1), axis=1)[:, None, None]
        # slope of E(x + t v) at t = 0 from a least-squares quadratic over |t| <= h
        h = 4e-3
        ts = np.linspace(-h, h, 33)
        Es = []
        for t in ts:
            xp = torch.from_numpy((x + t * v).astype(np.float32)).cuda()
            Es.append(model.energy_forces(xp, forces=False)[0].cpu().numpy())
        Es = np.array(Es)
        slope = np.polyfit(ts, Es, 2)[1]
        dd = np.sum(grad * v, axis=(1, 2)) / np.linspace(0.5, 1.5, M)
        np.testing.assert_allclose(dd, slope, rtol=3e-2, atol=3e-2 * np.abs(slope).max())
    finally:
        model.close()


def test_surrogate_dynamics_match_oracle(env):
    torch, pamd, S = env
    n, R, theta, dt, T, seed = 22, 96, 10, 0.001, 600.0, 31
    top = pi.make_chain(n, 2)
    x = pi.perturbed_positions(top, 64, 0.03, 5)
    model, q = _model_and_params(env, n, 128, 21, x)
    ctx = pamd.pamd_init(top, R, T, seed)
    try:
        x0, v0, _, _ = pamd.pamd_get_state(ctx)
        S.attach(ctx, model)
        pamd.pamd_propagate(ctx, theta, dt, T)
        x1, v1, E1, _ = pamd.pamd_get_state(ctx)
        sample = np.array([0, 41, R - 1])
        xo, vo, Eo = omlp.propagate(q, x0[sample], v0[sample], top.mass, theta, dt, T, 1.0, seed, 0,
                                    slots=sample)
        assert np.abs(x1[sample] - xo).max() < 1e-4
        assert np.abs(E1[sample] - Eo).max() <= 2e-2 * q["sigma_E"]
        # the population's energies are the model's energies of its positions
        Em, Fm = model.energy_forces(torch.from_numpy(x1.astype(np.float32)).cuda())
        np.testing.assert_allclose(E1, Em.cpu().numpy(), rtol=0, atol=1e-9 * q["sigma_E"])
        f, Ef = pamd.pamd_forces(ctx)
        np.testing.assert_allclose(f, Fm.cpu().numpy(), rtol=1e-5, atol=1e-3)
        # detaching restores the exact force field
        S.attach(ctx, None)
        f_exact, _ = pamd.pamd_forces(ctx)
        assert np.abs(f_exact - f).max() > 1.0
    finally:
        pamd.pamd_destroy(ctx)
        model.close()


def test_surrogate_anneal_graph_equals_stepwise_calls(env):
    """pamd_anneal with a force model runs as one CUDA graph in which each
    temperature's theta steps are a WHILE node (step kernel, four GEMMs and
    a loop counter per iteration).  It must reproduce, bit for bit, the same
    anneal issued as separate propagate / observables / resample calls (each
    queued step by step); a second launch continues with fresh counters, a
    new energy scale or detaching the model re-captures."""
    torch, pamd, S = env
    n, R, theta, dt, seed = 22, 300, 7, 0.001, 41
    top = pi.make_chain(n, 2)
    temps = pi.geometric_schedule(700.0, 500.0, 3)
    x = pi.perturbed_positions(top, 64, 0.03, 8)
    model, q = _model_and_params(env, n, 128, 9, x)
    a = pamd.pamd_init(top, R, temps[0], seed)
    b = pamd.pamd_init(top, R, temps[0], seed)
    try:
        S.attach(a, model)
        S.attach(b, model)
        l0 = pamd.pamd_launch_count(a)
        obs_a = pamd.pamd_anneal(a, temps, theta, dt)
        # every MD step ran: at least the step kernel and four GEMMs per step
        assert pamd.pamd_launch_count(a) - l0 >= len(temps) * theta * 5
        obs_b = []
        pamd.pamd_propagate(b, theta, dt, temps[0])
        obs_b.append(pamd.pamd_observables(b, temps[0]))
        for i in range(1, len(temps)):
            pamd.pamd_resample(b, temps[i - 1], temps[i], want_copies=False)
            pamd.pamd_propagate(b, theta, dt, temps[i])
            obs_b.append(pamd.pamd_observables(b, temps[i]))
        for u, w in zip(pamd.pamd_get_state(a), pamd.pamd_get_state(b)):
            np.testing.assert_array_equal(u, w)
        for oa, ob in zip(obs_a, obs_b):
            for k in oa:
                assert oa[k] == ob[k], k
        assert pamd.pamd_get_counters(a) == pamd.pamd_get_counters(b)
        # second launch of the same graph: fresh counters, still equal to the stepwise calls
        obs_a2 = pamd.pamd_anneal(a, temps, theta, dt)
        pamd.pamd_propagate(b, theta, dt, temps[0])
        ob0 = pamd.pamd_observables(b, temps[0])
        assert obs_a2[0]["e_pot"] == ob0["e_pot"] and obs_a2[0]["rg"] == ob0["rg"]
        assert obs_a2[-1]["e_pot"] != obs_a[-1]["e_pot"]
        # a new energy scale is seen by the next anneal (the graph is re-captured)
        p = model.get_params()
        p["mu_E"] = p["mu_E"] + 100.0
        model.set_params(p)
        c = pamd.pamd_init(top, R, temps[0], seed)
        try:
            S.attach(c, model)
            pamd.pamd_set_state(c, *pamd.pamd_get_state(a))
            pamd.pamd_set_counters(c, *pamd.pamd_get_counters(a))
            o1 = pamd.pamd_anneal(a, temps, theta, dt)
            o2 = pamd.pamd_anneal(c, temps, theta, dt)
            for k in o1[-1]:
                assert o1[-1][k] == o2[-1][k], k
        finally:
            pamd.pamd_destroy(c)
        # detaching restores the exact force field in the graph as well
        S.attach(a, None)
        e = pamd.pamd_init(top, R, temps[0], seed)
        try:
            pamd.pamd_set_state(e, *pamd.pamd_get_state(a))
            pamd.pamd_set_counters(e, *pamd.pamd_get_counters(a))
            oa = pamd.pamd_anneal(a, temps, theta, dt)
            oe = pamd.pamd_anneal(e, temps, theta, dt)
            for k in oa[-1]:
                assert oa[-1][k] == oe[-1][k], k
        finally:
            pamd.pamd_destroy(e)
    finally:
        pamd.pamd_destroy(a)
        pamd.pamd_destroy(b)
        model.close()


def test_training_gain_over_untrained_network(env):
    """What training buys: on exact data harvested by the GPU path, Adam lowers
    the held-out force error, and a PAMD anneal driven by the trained network
    reproduces the exact anneal's <E>(T) and <R_g>(T) far better than one
    driven by the same network untrained.  (Against the exact force field
    the surrogate gains no speed on this molecule: its force evaluation costs
    ~55x the flops; the benchmark reports both anneal times.)"""
    torch, pamd, S = env
    n = 22
    top = pi.make_chain(n, 1)
    temps = pi.geometric_schedule(1000.0, 300.0, 12)
    x, E, F = S.harvest(top, 1024, temps, 50, 0.001, 3)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    xt, Et, Ft = dev(x), dev(E), dev(F)
    n_train = (len(x) * 3) // 4
    trained = S.MLP(n, 128, seed=1)
    untrained = S.MLP(n, 128, seed=1)
    try:
        for m in (trained, untrained):
            m.fit_normalization(xt[:n_train], Et[:n_train])

        def force_rmse(m):
            _, Fp = m.energy_forces(xt[n_train:])
            return float(torch.sqrt(torch.mean((Fp - Ft[n_train:]) ** 2)))

        before = force_rmse(trained)
        hist = trained.train(xt[:n_train], Et[:n_train], Ft[:n_train], epochs=10, batch=256,
                             lam=1.0, lr=2e-3, lr_final=2e-4, report_every=50)
        after = force_rmse(trained)
        assert hist[-1][1] < 0.3 * hist[0][1]
        assert after < 0.5 * before, (before, after)

        # short anneals, identical seeds and schedule
        ta = pi.geometric_schedule(800.0, 500.0, 4)

        def anneal(model):
            ctx = pamd.pamd_init(top, 512, ta[0], 17)
            try:
                if model is not None:
                    S.attach(ctx, model)
                return pamd.pamd_anneal(ctx, ta, 100, 0.001)
            finally:
                pamd.pamd_destroy(ctx)

        ex, tr = anneal(None), anneal(trained)
        err = lambda o, key: max(abs(a[key] - b[key]) for a, b in zip(o, ex))
        try:
            un = anneal(untrained)
            un_e, un_r = err(un, "e_pot"), err(un, "rg")
        except pamd.PamdError:  # the untrained surface may not even stay finite
            un_e = un_r = float("inf")
        assert err(tr, "e_pot") < 0.5 * un_e, (err(tr, "e_pot"), un_e)
        assert err(tr, "rg") < 0.5 * un_r, (err(tr, "rg"), un_r)
    finally:
        trained.close()
        untrained.close()


def test_model_file_roundtrip(env, tmp_path):
    torch, _, S = env
    n = 22
    x = pi.perturbed_positions(pi.make_chain(n, 3), 32, 0.03, 7)
    model, _ = _model_and_params(env, n, 128, 5, x)
    path = str(tmp_path / "m.mlp")
    try:
        model.save(path)
        loaded = S.MLP.load(path)
        try:
            pa, pb = model.get_params(), loaded.get_params()
            for k in pa:
                np.testing.assert_array_equal(np.asarray(pa[k]), np.asarray(pb[k]))
            xt = torch.from_numpy(x.astype(np.float32)).cuda()
            Ea, Fa = model.energy_forces(xt)
            Eb, Fb = loaded.energy_forces(xt)
            np.testing.assert_array_equal(Ea.cpu().numpy(), Eb.cpu().numpy())
            np.testing.assert_array_equal(Fa.cpu().numpy(), Fb.cpu().numpy())
        finally:
            loaded.close()
        raw = bytearray(open(path, "rb").read())
        raw[-20] ^= 1
        open(path, "wb").write(bytes(raw))
        with pytest.raises(Exception):
            S.MLP.load(path)
    finally:
        model.close()
