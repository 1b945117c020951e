"""Pins of the coarse-grained mapping in the oracle (Eq. 9, 12, 14, 17)."""
import numpy as np
import pytest

import oracle
from paper_2603_01234_gb300 import inputs


def water_molecules(n_mol, box, seed):
    """n_mol rigid three-site molecules (masses 16, 1, 1) at random positions."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0, box, size=(n_mol, 3))
    off = np.array([[0.0, 0.0, 0.0], [0.96, 0.0, 0.0], [-0.24, 0.93, 0.0]])
    pos = (centres[:, None, :] + off[None]).reshape(-1, 3).T.copy()
    mass = np.tile([16.0, 1.0, 1.0], n_mol)
    start = np.arange(0, 3 * n_mol + 1, 3)
    atoms = np.arange(3 * n_mol)
    return pos, mass, start, atoms, centres, off


# Eq. 9 closed form: the mass-weighted centre of each molecule
def test_cg_centre_of_mass_closed_form():
    pos, mass, start, atoms, centres, off = water_molecules(20, 30.0, 1)
    bp, _, _ = oracle.cg_map(start, atoms, mass, pos, [30.0] * 3, [0, 0, 0])
    com_off = (np.array([16.0, 1.0, 1.0])[:, None] * off).sum(axis=0) / 18.0
    np.testing.assert_allclose(bp.T, centres + com_off, atol=1e-12)


# a molecule split across a periodic boundary maps to the same (wrapped) centre
def test_cg_periodic_unwrapping():
    L = 12.0
    pos, mass, start, atoms, centres, off = water_molecules(5, L, 2)
    pos[:, 3] = [L - 0.2, 5.0, 5.0]  # molecule 1 straddles x = 0 / L
    pos[:, 4] = pos[:, 3] + [0.96, 0.0, 0.0]
    pos[:, 5] = pos[:, 3] + [-0.24, 0.93, 0.0]
    shifted = pos.copy()
    shifted[0, 4] -= L  # the same configuration with one atom wrapped
    a, _, _ = oracle.cg_map(start, atoms, mass, pos, [L] * 3, [1, 1, 1])
    b, _, _ = oracle.cg_map(start, atoms, mass, shifted, [L] * 3, [1, 1, 1])
    np.testing.assert_allclose(a, b, atol=1e-12)
    expect = (16 * pos[:, 3] + pos[:, 4] + pos[:, 5]) / 18.0
    expect[0] %= L
    np.testing.assert_allclose(a[:, 1], expect, atol=1e-12)


# Eq. 12 / Eq. 14 with atomic forces and virials of an NEP evaluation: sums over
# groups, so bead forces sum to zero and bead virials sum to the total virial
def test_cg_force_and_virial_sums():
    model = inputs.random_model(seed=3, rc_radial=5.0, rc_angular=4.0)
    s = inputs.random_periodic(60, [14.0, 15.0, 16.0], seed=4, min_dist=1.3)
    r = oracle.compute(model, s)
    rng = np.random.default_rng(5)
    perm = rng.permutation(s.n)
    start = np.arange(0, s.n + 1, 4)  # 15 beads of 4 atoms
    _, bf, bw = oracle.cg_map(start, perm, np.ones(s.n), s.pos, s.box, s.pbc, r.force, r.virial)
    np.testing.assert_allclose(bf.sum(axis=1), 0.0, atol=1e-11)
    np.testing.assert_allclose(bw.sum(axis=1), r.virial_total, atol=1e-11)
    for I in range(15):
        np.testing.assert_allclose(bf[:, I], r.force[:, perm[4 * I:4 * I + 4]].sum(axis=1), atol=1e-14)
