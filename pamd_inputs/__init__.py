"""Seeded synthetic inputs for population-annealing molecular dynamics.

This module is shared by the CUDA library's tests and benchmarks and by the
FP64 oracle's tests.  It holds no arithmetic of the method itself: it only
draws the parameters of a synthetic peptide-like chain, builds a start
geometry, lays out temperature schedules and perturbs configurations for
tests.  Every random draw here uses numpy's PCG64 generator seeded by the
caller; the random numbers that the method itself draws (Langevin noise,
initial velocities, resampling uniforms) are NOT made here -- each side
implements Philox4x32-10 on its own.

Units: nm, ps, amu, elementary charge, K, kJ/mol, radians.

The chain recipe (all draws independent and uniform unless stated):
  * masses 12 amu;
  * bond (i, i+1): r0 ~ U(0.10, 0.15) nm, k = 2e5 kJ/mol/nm^2;
  * angle (i, i+1, i+2): theta0 ~ U(105, 120) degrees, k = 400 kJ/mol/rad^2;
  * dihedral (i..i+3): n uniform in {1, 2, 3}, k ~ U(0, 10) kJ/mol, phase 0;
  * LJ sigma ~ U(0.25, 0.35) nm, epsilon ~ U(0.1, 0.5) kJ/mol;
  * charges ~ N(0, 0.3) e, shifted so that they sum to zero;
  * 1-2 and 1-3 pairs excluded from the nonbonded sum, 1-4 pairs scaled 0.5
    (both Lennard-Jones and Coulomb);
  * start geometry: all-trans chain (every dihedral 180 degrees) placed by the
    natural-extension reference frame construction from r0 and theta0.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Topology",
    "make_chain",
    "make_harmonic_chain",
    "batched_chain_sizes",
    "geometric_schedule",
    "perturbed_positions",
    "gaussian_velocities",
    "random_energies",
]


@dataclass
class Topology:
    """Force-field description of one molecule (arrays are numpy, C-contiguous)."""

    n_atoms: int
    mass: np.ndarray      # [N] amu
    charge: np.ndarray    # [N] e
    sigma: np.ndarray     # [N] nm
    epsilon: np.ndarray   # [N] kJ/mol
    x0: np.ndarray        # [N,3] nm, start geometry
    bond: np.ndarray      # [nb,2] int32
    bond_r0: np.ndarray   # [nb] nm
    bond_k: np.ndarray    # [nb] kJ/mol/nm^2
    angle: np.ndarray     # [na,3] int32
    angle_t0: np.ndarray  # [na] rad
    angle_k: np.ndarray   # [na] kJ/mol/rad^2
    dihedral: np.ndarray  # [nd,4] int32
    dih_n: np.ndarray     # [nd] int32 multiplicity
    dih_k: np.ndarray     # [nd] kJ/mol
    dih_phase: np.ndarray  # [nd] rad
    excl: np.ndarray      # [ne,2] int32, pairs left out of the nonbonded sum
    pair14: np.ndarray    # [n14,2] int32, pairs whose nonbonded terms are scaled
    scale14_lj: float = 0.5
    scale14_coul: float = 0.5
    name: str = field(default="chain")

    def arrays(self):
        """Return every array field made C-contiguous with the dtype the C code expects."""
        f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
        return dict(
            mass=f64(self.mass), charge=f64(self.charge), sigma=f64(self.sigma),
            epsilon=f64(self.epsilon), x0=f64(self.x0).reshape(-1, 3),
            bond=i32(self.bond).reshape(-1, 2), bond_r0=f64(self.bond_r0), bond_k=f64(self.bond_k),
            angle=i32(self.angle).reshape(-1, 3), angle_t0=f64(self.angle_t0), angle_k=f64(self.angle_k),
            dihedral=i32(self.dihedral).reshape(-1, 4), dih_n=i32(self.dih_n), dih_k=f64(self.dih_k),
            dih_phase=f64(self.dih_phase), excl=i32(self.excl).reshape(-1, 2),
            pair14=i32(self.pair14).reshape(-1, 2),
        )


def _nerf_chain(r0: np.ndarray, t0: np.ndarray, dihedral_deg: float = 180.0) -> np.ndarray:
    """All-trans start geometry: place atom k+3 from atoms k..k+2, bond length r0[k+2],
    bond angle t0[k+1] and a fixed torsion (natural-extension reference frame)."""
    n = len(r0) + 1
    x = np.zeros((n, 3))
    if n == 1:
        return x
    x[1] = [r0[0], 0.0, 0.0]
    if n == 2:
        return x
    a = t0[0]
    # atom 2 in the xy plane, bond angle a at atom 1
    x[2] = x[1] + r0[1] * np.array([-np.cos(a), np.sin(a), 0.0])
    phi = np.deg2rad(dihedral_deg)
    for k in range(3, n):
        A, B, C = x[k - 3], x[k - 2], x[k - 1]
        bc = C - B
        bc /= np.linalg.norm(bc)
        nrm = np.cross(B - A, bc)
        nrm /= np.linalg.norm(nrm)
        m = np.stack([bc, np.cross(nrm, bc), nrm], axis=1)
        ang = t0[k - 2]
        d2 = r0[k - 1] * np.array([-np.cos(ang), np.sin(ang) * np.cos(phi), np.sin(ang) * np.sin(phi)])
        x[k] = C + m @ d2
    return x


def make_chain(n_atoms: int, seed: int, *, mass: float = 12.0) -> Topology:
    """Seeded linear peptide-like chain with the recipe in the module docstring."""
    if n_atoms < 1:
        raise ValueError("n_atoms must be >= 1")
    rng = np.random.default_rng(seed)
    n = n_atoms
    nb, na, nd = max(n - 1, 0), max(n - 2, 0), max(n - 3, 0)
    bond_r0 = rng.uniform(0.10, 0.15, nb)
    angle_t0 = np.deg2rad(rng.uniform(105.0, 120.0, na))
    dih_n = rng.integers(1, 4, nd).astype(np.int32)
    dih_k = rng.uniform(0.0, 10.0, nd)
    sigma = rng.uniform(0.25, 0.35, n)
    epsilon = rng.uniform(0.1, 0.5, n)
    charge = rng.normal(0.0, 0.3, n)
    charge -= charge.mean()
    idx = np.arange(n, dtype=np.int32)
    bond = np.stack([idx[:nb], idx[:nb] + 1], axis=1) if nb else np.zeros((0, 2), np.int32)
    angle = np.stack([idx[:na], idx[:na] + 1, idx[:na] + 2], axis=1) if na else np.zeros((0, 3), np.int32)
    dihedral = (np.stack([idx[:nd], idx[:nd] + 1, idx[:nd] + 2, idx[:nd] + 3], axis=1)
                if nd else np.zeros((0, 4), np.int32))
    excl = [(i, i + d) for d in (1, 2) for i in range(n - d)]
    excl = np.array(sorted(excl), dtype=np.int32).reshape(-1, 2)
    pair14 = np.array([(i, i + 3) for i in range(n - 3)], dtype=np.int32).reshape(-1, 2)
    x0 = _nerf_chain(bond_r0, angle_t0) if n > 1 else np.zeros((1, 3))
    return Topology(
        n_atoms=n, mass=np.full(n, float(mass)), charge=charge, sigma=sigma, epsilon=epsilon,
        x0=x0, bond=bond, bond_r0=bond_r0, bond_k=np.full(nb, 2.0e5),
        angle=angle, angle_t0=angle_t0, angle_k=np.full(na, 400.0),
        dihedral=dihedral, dih_n=dih_n, dih_k=dih_k, dih_phase=np.zeros(nd),
        excl=excl, pair14=pair14, name=f"chain{n}_s{seed}",
    )


def make_harmonic_chain(n_atoms: int, k: float, r0: float = 0.0, *, mass: float = 12.0,
                        seed: int = 0) -> Topology:
    """Bonds-only chain: harmonic springs (i, i+1) with rest length r0 and constant k.

    Every pair is excluded from the nonbonded sum and there are no angles or
    dihedrals, so each bond vector is an independent 3-D harmonic oscillator
    (for r0 = 0 an isotropic Gaussian).  The start geometry is a straight line
    with spacing max(r0, 0.1) nm, jittered by 0.01 nm from ``seed``.
    """
    n = n_atoms
    rng = np.random.default_rng(seed)
    idx = np.arange(n, dtype=np.int32)
    nb = n - 1
    bond = np.stack([idx[:nb], idx[:nb] + 1], axis=1)
    excl = np.array([(i, j) for i in range(n) for j in range(i + 1, n)], dtype=np.int32).reshape(-1, 2)
    x0 = np.zeros((n, 3))
    x0[:, 0] = np.arange(n) * max(r0, 0.1)
    x0 += rng.normal(0.0, 0.01, x0.shape)
    z = lambda s: np.zeros(s)
    return Topology(
        n_atoms=n, mass=np.full(n, float(mass)), charge=z(n), sigma=np.full(n, 0.3), epsilon=z(n),
        x0=x0, bond=bond, bond_r0=np.full(nb, float(r0)), bond_k=np.full(nb, float(k)),
        angle=np.zeros((0, 3), np.int32), angle_t0=z(0), angle_k=z(0),
        dihedral=np.zeros((0, 4), np.int32), dih_n=np.zeros(0, np.int32), dih_k=z(0), dih_phase=z(0),
        excl=excl, pair14=np.zeros((0, 2), np.int32), name=f"harmonic{n}",
    )


def batched_chain_sizes(n_mol: int = 16, seed: int = 7, lo: int = 20, hi: int = 200) -> list[int]:
    """Atom counts of the batched-uneven workload: N ~ U{lo..hi}, drawn with ``seed``."""
    rng = np.random.default_rng(seed)
    return [int(v) for v in rng.integers(lo, hi + 1, n_mol)]


def geometric_schedule(t_first: float, t_last: float, k_steps: int) -> np.ndarray:
    """Temperatures T_i = T_first * (T_last/T_first)^(i/K), i = 0..K (K+1 values)."""
    i = np.arange(k_steps + 1, dtype=np.float64)
    return t_first * (t_last / t_first) ** (i / max(k_steps, 1))


def perturbed_positions(top: Topology, n_rep: int, scale: float, seed: int) -> np.ndarray:
    """[n_rep, N, 3] copies of the start geometry with N(0, scale^2) jitter per coordinate."""
    rng = np.random.default_rng(seed)
    return top.x0[None, :, :] + rng.normal(0.0, scale, (n_rep, top.n_atoms, 3))


def gaussian_velocities(n_rep: int, n_atoms: int, scale: float, seed: int) -> np.ndarray:
    """[n_rep, N, 3] velocities N(0, scale^2) per component (test input, nm/ps)."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, (n_rep, n_atoms, 3))


def random_energies(n_rep: int, mean: float, spread: float, seed: int) -> np.ndarray:
    """[n_rep] energies N(mean, spread^2) in kJ/mol (test input for resampling)."""
    rng = np.random.default_rng(seed)
    return rng.normal(mean, spread, n_rep)
