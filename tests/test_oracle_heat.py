"""Pins of the oracle's heat current and HNEMD driving force (the thermal-conductivity
runs of Sec. III.B, following Fan et al. 2015 and 2019) against identities that
fix them independently of the per-particle virial code:

- the potential heat current of an open cluster equals
  sum_i r_i (F_i . v_i) + sum_i r_i dU_i/dt, with dU_i/dt by central finite
  differences of the site energies along the velocity field (this follows from
  J = d/dt sum_i r_i E_i; it fixes which index of W_i meets v_i);
- the driving forces sum to zero and add power F_e . J_pot;
- a driven NVE run gains exactly the energy integral of F_e . J_pot;
- F_e = 0 gives the undriven trajectory.
"""
import numpy as np
import pytest

import oracle
from paper_2603_01234_gb300 import inputs


def cluster_model():
    return inputs.random_model(n_types=2, n_desc_radial=3, n_desc_angular=2, n_basis_radial=5, n_basis_angular=5,
                               hidden=6, rc_radial=5.0, rc_angular=4.0, seed=31, scale=0.3)


def cluster(n=14, seed=32):
    s = inputs.random_cluster(n, seed=seed, box_len=8.0, min_dist=1.6, n_types=2)
    s.masses = np.array([12.0, 40.0])
    s.pos = s.pos - s.pos.mean(axis=1, keepdims=True)  # centred: small lever arms
    return s


def velocities(s, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((3, s.n)) * 0.01


def test_heat_current_equals_energy_moment_rate():
    m, s = cluster_model(), cluster()
    v = velocities(s, 33)
    r = oracle.compute(m, s)
    jpot, jkin = oracle.heat_current(s, v, r.site_energy, r.virial)
    # reference from site energies and forces only
    eps = 1e-4 / np.abs(v).max()
    up = oracle.compute(m, inputs.System(pos=s.pos + eps * v, types=s.types, box=s.box, pbc=s.pbc)).site_energy
    dn = oracle.compute(m, inputs.System(pos=s.pos - eps * v, types=s.types, box=s.box, pbc=s.pbc)).site_energy
    dUdt = (up - dn) / (2 * eps)
    fv = (r.force * v).sum(axis=0)
    ref = (s.pos * fv[None, :]).sum(axis=1) + (s.pos * dUdt[None, :]).sum(axis=1)
    scale = np.abs(s.pos * fv[None, :]).sum() + np.abs(s.pos * dUdt[None, :]).sum()
    assert np.abs(jpot - ref).max() <= 1e-7 * scale, (jpot, ref)
    # the transposed contraction is a different number (W_i is not symmetric)
    Wt = r.virial.reshape(3, 3, s.n).transpose(1, 0, 2).reshape(9, s.n)
    jt, _ = oracle.heat_current(s, v, r.site_energy, Wt)
    assert np.abs(jt - ref).max() > 1e3 * np.abs(jpot - ref).max()
    # convective part: sum_i (1/2 m v^2 + U_i) v_i
    mi = s.masses[s.types]
    Ei = 0.5 * mi * (v * v).sum(axis=0) / inputs.ACC_EV_A_AMU + r.site_energy
    np.testing.assert_allclose(jkin, (Ei[None, :] * v).sum(axis=1), rtol=1e-13, atol=1e-16)


def test_driving_force_momentum_and_power():
    m = inputs.random_model(n_types=1, hidden=10, rc_radial=6.0, rc_angular=4.0, seed=34, scale=0.2)
    s = inputs.water_small()
    r = oracle.compute(m, s)
    v = inputs.maxwell_boltzmann(s, 300.0, seed=35)  # one type: zero momentum means sum v = 0
    fe = np.array([0.3, -0.2, 0.5])
    fext = oracle.hnemd_force(fe, r.virial, np.zeros((3, s.n)))
    assert np.abs(fext.sum(axis=1)).max() <= 1e-12 * np.abs(fext).sum()
    jpot, _ = oracle.heat_current(s, v, r.site_energy, r.virial)
    power = (fext * v).sum()
    assert power == pytest.approx(fe @ jpot, rel=1e-10)
    # it is added to the force, not substituted
    f2 = oracle.hnemd_force(fe, r.virial, r.force)
    np.testing.assert_allclose(f2 - r.force, fext, atol=1e-14)


@pytest.fixture(scope="module")
def driven_runs():
    m = inputs.random_model(n_types=1, hidden=10, rc_radial=6.0, rc_angular=4.0, seed=36, scale=0.2)
    s = inputs.water_small()
    v0 = inputs.maxwell_boltzmann(s, 300.0, seed=37)
    r0 = oracle.compute(m, s)
    fe = np.array([0.0, 0.1, 0.25])
    f0 = oracle.hnemd_force(fe, r0.virial, r0.force)
    j0, _ = oracle.heat_current(s, v0, r0.site_energy, r0.virial)
    steps, dt = 60, 0.5
    drv = oracle.md(m, s, s.pos, v0, f0, steps, dt, fe=fe)
    nve = oracle.md(m, s, s.pos, v0, r0.force, steps, dt)
    zero = oracle.md(m, s, s.pos, v0, r0.force, steps, dt, fe=np.zeros(3))
    ke0 = 0.5 * s.masses[0] * (v0 * v0).sum() / inputs.ACC_EV_A_AMU
    return dict(s=s, fe=fe, dt=dt, h0=r0.energy + ke0, j0=j0, v0=v0, drv=drv, nve=nve, zero=zero)


def test_driven_run_gains_the_power_integral(driven_runs):
    d = driven_runs
    _, vel, _, thermo, heat = d["drv"]
    H = thermo.sum(axis=1)
    p = np.concatenate([[d["fe"] @ d["j0"]], heat[:, :3] @ d["fe"]])
    work = np.concatenate([[0.0], np.cumsum(0.5 * d["dt"] * (p[1:] + p[:-1]))])
    dH = np.concatenate([[0.0], H - d["h0"]])
    nve_dH = np.abs(d["nve"][3].sum(axis=1) - d["h0"]).max()
    assert np.abs(work).max() > 50 * nve_dH  # the drive dominates the integrator's error
    assert np.abs(dH - work).max() <= 0.02 * np.abs(work).max() + 2 * nve_dH
    assert np.abs(vel.sum(axis=1)).max() <= 1e-12 * np.abs(vel).sum()  # momentum stays zero


def test_zero_field_is_the_plain_trajectory(driven_runs):
    d = driven_runs
    np.testing.assert_array_equal(d["zero"][0], d["nve"][0])
    np.testing.assert_array_equal(d["zero"][1], d["nve"][1])
    np.testing.assert_array_equal(d["zero"][3], d["nve"][3])


def test_running_kappa_units():
    """kappa = <J> / (T V F_e); 1 eV A/fs / (K A^3 A^-1) = 1.602176634e6 W/(m K)."""
    from paper_2603_01234_gb300 import transport
    heat = np.zeros((4, 6))
    heat[:, 2] = [1.0, 3.0, 2.0, 2.0]  # J_pot,z
    heat[:, 5] = 10.0                   # J_kin,z
    k = transport.running_kappa(heat, temperature=300.0, volume=1000.0, fe=[0.0, 0.0, 1e-3], axis=2)
    np.testing.assert_allclose(k, np.array([1.0, 2.0, 2.0, 2.0]) / (300.0 * 1000.0 * 1e-3) * 1.602176634e6)
    k2 = transport.running_kappa(heat, 300.0, 1000.0, [0.0, 0.0, 1e-3], axis=2, include_kinetic=True, dof_scale=60)
    np.testing.assert_allclose(k2, 60 * (np.array([1.0, 2.0, 2.0, 2.0]) + 10.0) / 300.0 * 1.602176634e6)
    with pytest.raises(ValueError):
        transport.running_kappa(heat, 300.0, 1000.0, [1e-3, 0.0, 1e-3], axis=2)
