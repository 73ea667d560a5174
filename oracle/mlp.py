"""FP64 CPU oracle of the MLP energy surrogate -- TEST INFRASTRUCTURE.

Only the test suite and the benchmark's CPU legs use this module.  It is plain
numpy in float64, written from the definition of the surrogate:

  features   g_p = 1 / r_ij for every pair p = (i, j), i < j, in row order
             (i = 0: j = 1..N-1, then i = 1, ...), normalised a = (g - mu) / sd
  layer 1    z1 = W1 a + b1,  h1 = silu(z1)          (W1: [H, P])
  layer 2    z2 = W2 h1 + b2, h2 = silu(z2)          (W2: [H, H])
  output     e  = w3 . h2 + b3   (normalised energy; E = sigma_E e + mu_E)
  forces     F_k = -dE/dx_k = -sigma_E sum_p (de/dg_p) dg_p/dx_k,
             dg_p/dx_i = -(x_i - x_j) / r^3 = -dg_p/dx_j,
  with silu(z) = z s(z), s the logistic function.

Training loss of one sample (normalised units, forces divided by sigma_E):
  L = (e - e_ref)^2 + lam / (3N) sum_k |f_k - f_ref,k|^2,   f = F / sigma_E.
Its gradient with respect to the weights: the energy term by ordinary
backpropagation; the force term through the directional derivative of e
along nu = dL/d(de/da) (forward tangent pass), differentiated in reverse.
"""
from __future__ import annotations

import numpy as np


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def d2silu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    ds = s * (1.0 - s)
    return ds * (2.0 + z * (1.0 - 2.0 * s))


def pair_index(n):
    """(i, j) arrays of all pairs i < j in row order."""
    i, j = np.triu_indices(n, 1)
    return i, j


def features(x):
    """Inverse pair distances g [M, P] of configurations x [M, N, 3]."""
    x = np.asarray(x, dtype=np.float64)
    i, j = pair_index(x.shape[1])
    d = x[:, i, :] - x[:, j, :]
    return 1.0 / np.sqrt(np.sum(d * d, axis=-1))


def init_params(n_atoms, hidden=512, seed=0):
    """Random weights (He-like scale) and identity normalisation."""
    rng = np.random.default_rng(seed)
    P = n_atoms * (n_atoms - 1) // 2
    return {
        "W1": rng.normal(0.0, np.sqrt(1.0 / P), (hidden, P)),
        "b1": np.zeros(hidden),
        "W2": rng.normal(0.0, np.sqrt(1.0 / hidden), (hidden, hidden)),
        "b2": np.zeros(hidden),
        "w3": rng.normal(0.0, np.sqrt(1.0 / hidden), hidden),
        "b3": 0.0,
        "mu": np.zeros(P),
        "sd": np.ones(P),
        "mu_E": 0.0,
        "sigma_E": 1.0,
    }


def forward(p, x):
    """Energies E [M] (kJ/mol) and the intermediates of configurations x [M, N, 3]."""
    g = features(x)
    a = (g - p["mu"]) / p["sd"]
    z1 = a @ p["W1"].T + p["b1"]
    h1 = silu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = silu(z2)
    e = h2 @ p["w3"] + p["b3"]
    return p["sigma_E"] * e + p["mu_E"], dict(g=g, a=a, z1=z1, h1=h1, z2=z2, h2=h2, e=e)


def pair_jacobian_apply(x, gamma_g):
    """sum_p gamma_p dg_p/dx_k for each atom k: x [M,N,3], gamma_g [M,P] -> [M,N,3]."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[1]
    i, j = pair_index(n)
    d = x[:, i, :] - x[:, j, :]
    r = np.sqrt(np.sum(d * d, axis=-1))
    c = (-gamma_g / r ** 3)[..., None] * d          # gamma * dg/dx_i
    out = np.zeros_like(x)
    np.add.at(out, (slice(None), i), c)
    np.add.at(out, (slice(None), j), -c)
    return out


def energy_forces(p, x):
    """E [M] and F [M, N, 3] by the analytic backward pass."""
    E, c = forward(p, x)
    d2 = p["w3"] * dsilu(c["z2"])
    d1 = (d2 @ p["W2"]) * dsilu(c["z1"])
    ga = d1 @ p["W1"]                                 # de/da
    gg = ga / p["sd"]                                 # de/dg
    F = -p["sigma_E"] * pair_jacobian_apply(x, gg)
    return E, F


def loss_and_grads(p, x, E_ref, F_ref, lam):
    """Mean loss over the M samples and its gradient dict (W1, b1, W2, b2, w3, b3)."""
    M, n = x.shape[0], x.shape[1]
    E, c = forward(p, x)
    sE = p["sigma_E"]
    e_ref = (np.asarray(E_ref) - p["mu_E"]) / sE
    s1, s2 = dsilu(c["z1"]), dsilu(c["z2"])
    d2 = p["w3"] * s2                                 # [M, H]
    W2t_d2 = d2 @ p["W2"]                             # W2^T delta2, [M, H]
    d1 = W2t_d2 * s1
    ga = d1 @ p["W1"]                                 # de/da [M, P]
    gg = ga / p["sd"]
    f = -pair_jacobian_apply(x, gg)                   # normalised forces F / sigma_E
    f_ref = np.asarray(F_ref) / sE
    de = c["e"] - e_ref
    df = f - f_ref
    L = np.mean(de ** 2 + lam / (3 * n) * np.sum(df ** 2, axis=(1, 2)))
    # --- energy term: e_bar = dL/de
    e_bar = 2.0 * de / M
    # --- force term: u = dL/df, nu_g = dL/d(de/dg) = -J u, nu_a = nu_g / sd
    u = 2.0 * lam / (3 * n) * df / M
    nu_g = -pair_jacobian_apply_T(x, u)
    nu_a = nu_g / p["sd"]
    # tangent pass along nu_a
    zd1 = nu_a @ p["W1"].T
    hd1 = zd1 * s1
    zd2 = hd1 @ p["W2"].T
    hd2 = zd2 * s2
    # reverse over the tangent pass and the primal it reads
    z2_bar = e_bar[:, None] * d2 + p["w3"] * zd2 * d2silu(c["z2"])
    h1_bar = z2_bar @ p["W2"]
    z1_bar = h1_bar * s1 + W2t_d2 * zd1 * d2silu(c["z1"])
    g = {
        "w3": e_bar @ c["h2"] + np.sum(hd2, axis=0),
        "b3": float(np.sum(e_bar)),
        "W2": z2_bar.T @ c["h1"] + d2.T @ hd1,
        "b2": np.sum(z2_bar, axis=0),
        "W1": z1_bar.T @ c["a"] + d1.T @ nu_a,
        "b1": np.sum(z1_bar, axis=0),
    }
    return L, g


def pair_jacobian_apply_T(x, u):
    """J u for J = dg/dx: (J u)_p = dg_p/dx_i . u_i + dg_p/dx_j . u_j, [M, P]."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[1]
    i, j = pair_index(n)
    d = x[:, i, :] - x[:, j, :]
    r = np.sqrt(np.sum(d * d, axis=-1))
    dgi = -d / r[..., None] ** 3
    return np.sum(dgi * (u[:, i, :] - u[:, j, :]), axis=-1)


def propagate(p, x, v, masses, theta, dt, T, gamma, seed, step0, mol=0, slots=None):
    """theta BAOAB Langevin steps of configurations x, v [R, N, 3] with the
    surrogate's forces (FP64): the integrator and noise stream of the exact
    oracle (B, A, O, A, new forces, B; noise from Philox(seed; atom, slot,
    step0 + s, NOISE | mol << 8)).  Returns (x, v, E)."""
    from . import normal3
    kB = 0.008314462618
    x = np.array(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    R, n = x.shape[0], x.shape[1]
    slots = np.arange(R) if slots is None else np.asarray(slots)
    im = 1.0 / np.asarray(masses, dtype=np.float64)
    c1 = np.exp(-gamma * dt)
    sdv = np.sqrt((1.0 - c1 * c1) * kB * T * im)
    E, F = energy_forces(p, x)
    for s in range(theta):
        z = np.array([[normal3(seed, i, int(slots[r]), step0 + s, mol << 8) for i in range(n)]
                      for r in range(R)])
        v += 0.5 * dt * F * im[None, :, None]          # B
        x += 0.5 * dt * v                               # A
        v = c1 * v + sdv[None, :, None] * z             # O
        x += 0.5 * dt * v                               # A
        E, F = energy_forces(p, x)
        v += 0.5 * dt * F * im[None, :, None]          # B
    return x, v, E
