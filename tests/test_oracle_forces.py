"""Pins of the oracle's force field against closed forms and invariants.

Each test fixes a property that a plausible slip would break:
finite differences (force/energy consistency, sign of every term), the
two-atom Lennard-Jones minimum (Lorentz-Berthelot mixing: position and
depth), Coulomb's law for two charges, 1-4 scaling, exclusions, Newton's
third law, rotation/translation invariance, the IUPAC torsion sign, and
the minima/maxima of each bonded term.
"""
import math

import numpy as np
import pytest

import pamd_inputs as pi

KE = 138.935458


def _two_atoms(s1, s2, e1, e2, q1=0.0, q2=0.0):
    top = pi.make_chain(2, 0)
    top.sigma = np.array([s1, s2]); top.epsilon = np.array([e1, e2])
    top.charge = np.array([q1, q2])
    top.bond = np.zeros((0, 2), np.int32); top.bond_r0 = np.zeros(0); top.bond_k = np.zeros(0)
    top.excl = np.zeros((0, 2), np.int32)
    return top


def _fd_forces(orc, top, x, h=1e-6):
    fd = np.zeros_like(x)
    for i in range(x.shape[0]):
        for c in range(3):
            xp = x.copy(); xp[i, c] += h
            xm = x.copy(); xm[i, c] -= h
            fd[i, c] = -(orc.energy_forces(top, xp)[0] - orc.energy_forces(top, xm)[0]) / (2 * h)
    return fd


@pytest.mark.parametrize("n,seed", [(4, 1), (12, 2), (22, 3)])
def test_forces_match_finite_differences(orc, n, seed):
    top = pi.make_chain(n, seed)
    # give dihedrals nonzero phases so the torsion sign enters the energy
    top.dih_phase = np.linspace(0.3, 2.0, len(top.dih_phase))
    x = pi.perturbed_positions(top, 1, 0.02, seed + 10)[0]
    e, f, terms = orc.energy_forces(top, x)
    assert abs(e - terms.sum()) < 1e-9 * max(1.0, abs(e))
    fd = _fd_forces(orc, top, x)
    assert np.abs(fd - f).max() <= 1e-6 * np.abs(f).max() + 1e-6


def test_lj_minimum_lorentz_berthelot(orc):
    s1, s2, e1, e2 = 0.26, 0.34, 0.12, 0.45
    top = _two_atoms(s1, s2, e1, e2)
    rmin = 2 ** (1 / 6) * 0.5 * (s1 + s2)
    x = np.array([[0.0, 0.0, 0.0], [rmin, 0.0, 0.0]])
    e, f, _ = orc.energy_forces(top, x)
    assert abs(e + math.sqrt(e1 * e2)) < 1e-12
    assert np.abs(f).max() < 1e-9
    # the energy crosses zero at r = sigma_ij
    x[1, 0] = 0.5 * (s1 + s2)
    assert abs(orc.energy_forces(top, x)[0]) < 1e-12
    # repulsive inside, attractive outside the minimum
    x[1, 0] = 0.9 * rmin
    assert orc.energy_forces(top, x)[1][1, 0] > 0
    x[1, 0] = 1.2 * rmin
    assert orc.energy_forces(top, x)[1][1, 0] < 0


def test_coulomb_two_charges(orc):
    top = _two_atoms(0.3, 0.3, 0.0, 0.0, 0.4, -0.7)
    r = 0.8
    x = np.array([[0.1, 0.2, 0.3], [0.1, 0.2 + r, 0.3]])
    e, f, terms = orc.energy_forces(top, x)
    assert abs(e - KE * 0.4 * (-0.7) / r) < 1e-12
    # opposite charges attract: force on atom 1 points back towards atom 0
    assert abs(f[1, 1] - KE * 0.4 * 0.7 * (-1.0) / r**2) < 1e-10
    assert abs(terms[3]) < 1e-15


def test_pair14_scaling_and_exclusions(orc):
    # 4-atom chain with bonded terms switched off: only the 1-4 pair interacts
    top = pi.make_chain(4, 5)
    top.bond_k[:] = 0; top.angle_k[:] = 0; top.dih_k[:] = 0
    s03 = 0.5 * (top.sigma[0] + top.sigma[3])
    e03 = math.sqrt(top.epsilon[0] * top.epsilon[3])
    x = np.array([[0.0, 0, 0], [0.1, 0.3, 0], [0.2, 0.5, 0.1], [2 ** (1 / 6) * s03, 0, 0]])
    top.charge[:] = 0.0
    e, f, terms = orc.energy_forces(top, x)
    assert abs(terms[3] + 0.5 * e03) < 1e-12       # depth scaled by 0.5
    assert np.abs(f).max() < 1e-9                   # still a minimum
    # exclusions: moving the 1-2 and 1-3 partners arbitrarily changes nothing
    x2 = x.copy(); x2[1] = [0.001, 0.0, 0.0]; x2[2] = [0.0, 0.001, 0.0]
    assert abs(orc.energy_forces(top, x2)[2][3] - terms[3]) < 1e-12
    # 1-4 Coulomb scaled by 0.5 as well
    top.charge[:] = [0.5, 0.0, 0.0, -0.5]
    top.epsilon[:] = 0.0
    r = 0.9
    x3 = x.copy(); x3[3] = [r, 0, 0]
    assert abs(orc.energy_forces(top, x3)[2][4] - 0.5 * KE * 0.5 * (-0.5) / r) < 1e-12


def test_newton_and_rigid_motion_invariance(orc):
    top = pi.make_chain(30, 9)
    x = pi.perturbed_positions(top, 1, 0.02, 4)[0]
    e, f, _ = orc.energy_forces(top, x)
    assert np.abs(f.sum(0)).max() < 1e-9 * np.abs(f).max()
    # torque-free: sum r x F = 0 for an isolated molecule
    assert np.abs(np.cross(x, f).sum(0)).max() < 1e-8 * np.abs(f).max()
    rng = np.random.default_rng(0)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    xr = x @ q.T + np.array([1.0, -2.0, 0.5])
    er, fr, _ = orc.energy_forces(top, xr)
    assert abs(er - e) < 1e-9 * abs(e)
    assert np.abs(fr - f @ q.T).max() < 1e-8 * np.abs(f).max()


def test_dihedral_iupac_sign(orc):
    # looking down j->k (the +z axis), the rear bond k->l at +alpha
    # counter-clockwise seen from +z is a positive torsion
    for alpha in (0.0, 0.7, 2.0, -1.1, math.pi):
        xi, xj, xk = [1.0, 0, 0], [0.0, 0, 0], [0.0, 0, 1.0]
        xl = [math.cos(alpha), math.sin(alpha), 1.0]
        phi = orc.dihedral_angle(xi, xj, xk, xl)
        assert abs(math.remainder(phi - alpha, 2 * math.pi)) < 1e-12


def test_bonded_terms_closed_forms(orc):
    top = pi.make_chain(4, 1)
    top.epsilon[:] = 0; top.charge[:] = 0
    # cis (phi = 0) and trans (phi = pi) for n = 1: E = 2k and 0
    top.bond_k[:] = 0; top.angle_k[:] = 0
    top.dih_n[:] = 1; top.dih_k[:] = 3.5
    cis = np.array([[1.0, 0, 0], [0, 0, 0], [0, 0, 1.0], [1.0, 0, 1.0]])
    trans = np.array([[1.0, 0, 0], [0, 0, 0], [0, 0, 1.0], [-1.0, 0, 1.0]])
    assert abs(orc.energy_forces(top, cis)[2][2] - 7.0) < 1e-12
    assert abs(orc.energy_forces(top, trans)[2][2]) < 1e-12
    # n = 3: maxima at phi = 0, 120, 240 degrees
    top.dih_n[:] = 3
    for a in (0.0, 2 * math.pi / 3):
        g = np.array([[1.0, 0, 0], [0, 0, 0], [0, 0, 1.0], [math.cos(a), math.sin(a), 1.0]])
        assert abs(orc.energy_forces(top, g)[2][2] - 7.0) < 1e-12
    # bond and angle at their rest values: zero energy and force
    top = pi.make_chain(3, 2)
    top.epsilon[:] = 0; top.charge[:] = 0
    t0, r0a, r0b = top.angle_t0[0], top.bond_r0[0], top.bond_r0[1]
    x = np.array([[r0a, 0, 0], [0, 0, 0], [r0b * math.cos(t0), r0b * math.sin(t0), 0]])
    e, f, terms = orc.energy_forces(top, x)
    assert abs(e) < 1e-12 and np.abs(f).max() < 1e-8
    # stretch bond 0 by d: E = k d^2 / 2
    d = 0.01
    x[0, 0] += d
    assert abs(orc.energy_forces(top, x)[2][0] - 0.5 * top.bond_k[0] * d * d) < 1e-9
    # bend: rotate atom 2 by delta about z; E = k delta^2 / 2
    x[0, 0] -= d
    dl = 0.05
    x[2] = [r0b * math.cos(t0 + dl), r0b * math.sin(t0 + dl), 0]
    assert abs(orc.energy_forces(top, x)[2][1] - 0.5 * top.angle_k[0] * dl * dl) < 1e-9


def test_generator_recipe(orc):
    top = pi.make_chain(75, 1)
    assert abs(top.charge.sum()) < 1e-12
    assert top.bond_r0.min() >= 0.10 and top.bond_r0.max() <= 0.15
    assert np.rad2deg(top.angle_t0).min() >= 105 and np.rad2deg(top.angle_t0).max() <= 120
    assert set(np.unique(top.dih_n)) <= {1, 2, 3}
    # the start geometry realises r0, theta0 and all-trans torsions
    x = top.x0
    r = np.linalg.norm(x[1:] - x[:-1], axis=1)
    np.testing.assert_allclose(r, top.bond_r0, rtol=1e-12)
    phis = [orc.dihedral_angle(*x[k:k + 4]) for k in range(72)]
    assert np.allclose(np.abs(phis), math.pi, atol=1e-9)
    # no clashes: every non-excluded pair at least 0.25 nm apart
    d = np.linalg.norm(x[:, None] - x[None], axis=-1)
    iu = np.triu_indices(75, 3)
    assert d[iu].min() > 0.25
