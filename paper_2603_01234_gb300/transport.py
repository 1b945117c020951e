"""Thermal conductivity from HNEMD heat-current rows (Sec. III.B; the method of
Fan et al., Phys. Rev. B 99, 064308, 2019).

Under a driving-force parameter F_e the non-equilibrium heat current responds
linearly, <J_a> = T V kappa_ab Fe_b, so the running time average of the rows that
nep_md_step_hnemd writes gives kappa(t).  Host post-processing only.
"""
from __future__ import annotations

import numpy as np

# eV Angstrom / fs / (K Angstrom^3 Angstrom^-1) in W / (m K)
EV_PER_FS_A_K_TO_SI = 1.602176634e-19 / (1e-15 * 1e-10)


def running_kappa(heat, temperature, volume, fe, axis, include_kinetic=False, dof_scale=1.0):
    """Running kappa_{axis, b} in W/(m K) after each row of `heat` [rows][6]
    (interval averages of J_pot, J_kin in eV Angstrom / fs), for a driving force
    fe[3] (1/Angstrom) along one axis b (the only nonzero component), the
    temperature (K) and volume (Angstrom^3).  `dof_scale` multiplies the result
    (the paper scales coarse-grained values by the atoms per bead)."""
    heat = np.asarray(heat, dtype=np.float64)
    fe = np.asarray(fe, dtype=np.float64)
    nz = np.flatnonzero(fe)
    if nz.size != 1:
        raise ValueError("fe must have exactly one nonzero component")
    j = heat[:, axis] + (heat[:, 3 + axis] if include_kinetic else 0.0)
    avg = np.cumsum(j) / np.arange(1, j.size + 1)
    return dof_scale * avg / (temperature * volume * fe[nz[0]]) * EV_PER_FS_A_K_TO_SI
