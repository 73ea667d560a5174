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


def test_surrogate_dynamics_reduces_to_exact_oracle_without_forces(orc):
    """With W1 = 0 the surrogate exerts no force; a bonds-only chain with k = 0
    has none either, so both integrators must produce the same trajectory from
    the same noise stream (pins the B-A-O-A-B order, the O coefficients and the
    Philox counters of the surrogate integrator)."""
    n, R = 5, 3
    p = _small(n=n, hidden=4)
    p["W1"][:] = 0.0
    top = pi.make_harmonic_chain(n, 0.0, 0.0)
    rng = np.random.default_rng(4)
    x0 = top.x0[None] + rng.normal(0, 0.02, (R, n, 3))
    v0 = rng.normal(0, 0.5, (R, n, 3))
    slots = np.array([0, 5, 9])
    xs, vs, _ = mlp.propagate(p, x0, v0, top.mass, 4, 0.002, 400.0, 2.0, 99, 7, mol=1, slots=slots)
    xo, vo, _ = orc.propagate(top, x0, v0, 4, 0.002, 400.0, 2.0, 99, 7, mol=1, slots=slots)
    np.testing.assert_allclose(xs, xo, rtol=0, atol=1e-13)
    np.testing.assert_allclose(vs, vo, rtol=0, atol=1e-12)


def test_surrogate_nve_energy_error_scales_with_dt_squared():
    """gamma = 0: velocity Verlet on the surrogate surface; the total-energy
    error after a fixed time shrinks ~4x when dt halves (second order)."""
    n = 6
    x0 = _configs(n, 1, 12)
    p = mlp.init_params(n, 8, 11)
    p["mu"] = mlp.features(x0)[0]
    p["sd"] = np.full(n * (n - 1) // 2, 0.5)
    masses = np.full(n, 12.0)
    v0 = np.random.default_rng(3).normal(0, 0.3, (1, n, 3))

    def drift(dt, steps):
        E0, _ = mlp.energy_forces(p, x0)
        x, v, E = mlp.propagate(p, x0, v0, masses, steps, dt, 300.0, 0.0, 1, 0)
        k0 = 0.5 * np.sum(masses[None, :, None] * v0 ** 2)
        k1 = 0.5 * np.sum(masses[None, :, None] * v ** 2)
        return abs((E[0] + k1) - (E0[0] + k0))

    d1, d2 = drift(0.004, 25), drift(0.002, 50)
    assert d1 > 0 and 2.5 < d1 / d2 < 6.0, (d1, d2)
