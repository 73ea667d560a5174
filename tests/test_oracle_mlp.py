"""Pins of the FP64 MLP surrogate oracle (oracle/mlp.py).

* Forces equal minus the finite-difference gradient of the energy.
* The loss gradient equals central finite differences of the loss for
  sampled weights of every parameter block (energy and force terms).
* Special cases: with W1 = 0 the energy is constant and forces vanish; with
  the force weight lam = 0 the gradient is plain backpropagation of the
  energy term, and the two terms add linearly.
* Features are inverse distances in row order, invariant under rigid motion.
"""
import numpy as np
import pytest

import pamd_inputs as pi
from oracle import mlp


def _small(n=6, hidden=7, seed=1):
    p = mlp.init_params(n, hidden, seed)
    rng = np.random.default_rng(seed + 1)
    P = n * (n - 1) // 2
    p["b1"] = rng.normal(0, 0.3, hidden)
    p["b2"] = rng.normal(0, 0.3, hidden)
    p["mu"] = rng.uniform(0.5, 2.0, P)
    p["sd"] = rng.uniform(0.5, 2.0, P)
    p["mu_E"], p["sigma_E"] = -3.0, 2.5
    p["W1"] *= 3.0
    return p


def _configs(n, m, seed):
    top = pi.make_chain(n, seed)
    return pi.perturbed_positions(top, m, 0.03, seed)


def test_features_row_order_and_invariance():
    x = np.array([[[0, 0, 0], [1, 0, 0], [0, 2, 0], [0, 0, 4.0]]])
    np.testing.assert_allclose(mlp.features(x)[0],
                               [1, 0.5, 0.25, 1 / np.sqrt(5), 1 / np.sqrt(17), 1 / np.sqrt(20)])
    y = _configs(8, 2, 3)
    rng = np.random.default_rng(0)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    np.testing.assert_allclose(mlp.features(y @ q.T + 1.5), mlp.features(y), rtol=1e-12)


def test_forces_are_minus_energy_gradient():
    p = _small()
    x = _configs(6, 3, 4)
    E, F = mlp.energy_forces(p, x)
    h = 1e-6
    for m in range(3):
        for k in range(6):
            for c in range(3):
                xp = x.copy(); xp[m, k, c] += h
                xm = x.copy(); xm[m, k, c] -= h
                fd = -(mlp.forward(p, xp)[0][m] - mlp.forward(p, xm)[0][m]) / (2 * h)
                assert abs(fd - F[m, k, c]) <= 1e-6 * max(1.0, abs(F[m, k, c]))


@pytest.mark.parametrize("lam", [0.0, 0.7])
def test_loss_gradient_matches_finite_differences(lam):
    p = _small(seed=3)
    x = _configs(6, 4, 5)
    rng = np.random.default_rng(9)
    E_ref = rng.normal(-3, 2, 4)
    F_ref = rng.normal(0, 5, (4, 6, 3))
    L, g = mlp.loss_and_grads(p, x, E_ref, F_ref, lam)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "w3", "b3"):
        arr = np.atleast_1d(p[name])
        flat = arr.reshape(-1)
        picks = rng.choice(flat.size, size=min(6, flat.size), replace=False)
        for idx in picks:
            q = {k: (np.array(v, copy=True) if isinstance(v, np.ndarray) else v) for k, v in p.items()}
            qa = np.atleast_1d(q[name]).reshape(-1)
            qa[idx] += h
            q[name] = qa.reshape(np.shape(p[name])) if np.ndim(p[name]) else float(qa[0])
            Lp, _ = mlp.loss_and_grads(q, x, E_ref, F_ref, lam)
            qa[idx] -= 2 * h
            q[name] = qa.reshape(np.shape(p[name])) if np.ndim(p[name]) else float(qa[0])
            Lm, _ = mlp.loss_and_grads(q, x, E_ref, F_ref, lam)
            fd = (Lp - Lm) / (2 * h)
            an = np.atleast_1d(g[name]).reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (name, idx, fd, an)


def test_special_cases():
    p = _small()
    x = _configs(6, 2, 7)
    p["W1"][:] = 0.0
    E, F = mlp.energy_forces(p, x)
    assert np.allclose(E, E[0]) and np.abs(F).max() == 0.0
    # the loss gradient is linear in the two terms
    p = _small(seed=5)
    rng = np.random.default_rng(2)
    E_ref, F_ref = rng.normal(0, 1, 2), rng.normal(0, 3, (2, 6, 3))
    _, g0 = mlp.loss_and_grads(p, x, E_ref, F_ref, 0.0)
    _, g1 = mlp.loss_and_grads(p, x, E_ref, F_ref, 1.0)
    _, g2 = mlp.loss_and_grads(p, x, E_ref, F_ref, 2.0)
    for k in g0:
        np.testing.assert_allclose(np.asarray(g2[k]) - np.asarray(g1[k]),
                                   np.asarray(g1[k]) - np.asarray(g0[k]), rtol=1e-9, atol=1e-12)
