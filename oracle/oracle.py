"""ctypes wrapper of the FP64 C oracle (test infrastructure only).

The functions take numpy arrays in the same layouts as the CUDA library's C ABI
(positions SoA [3][n], virial [9][n] row-major alpha,beta) and return numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from .build import build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i, p = C.c_double, C.c_int, C.c_void_p
        _lib.oracle_fc.argtypes = [d, d]
        _lib.oracle_fc.restype = d
        _lib.oracle_dfc.argtypes = [d, d]
        _lib.oracle_dfc.restype = d
        _lib.oracle_fk.argtypes = [i, d, d]
        _lib.oracle_fk.restype = d
        _lib.oracle_dfk.argtypes = [i, d, d]
        _lib.oracle_dfk.restype = d
        _lib.oracle_chebyshev.argtypes = [i, d]
        _lib.oracle_chebyshev.restype = d
        _lib.oracle_dchebyshev.argtypes = [i, d]
        _lib.oracle_dchebyshev.restype = d
        _lib.oracle_gn.argtypes = [p, i, d, d]
        _lib.oracle_gn.restype = d
        _lib.oracle_dgn.argtypes = [p, i, d, d]
        _lib.oracle_dgn.restype = d
        _lib.oracle_legendre.argtypes = [i, d]
        _lib.oracle_legendre.restype = d
        _lib.oracle_dlegendre.argtypes = [i, d]
        _lib.oracle_dlegendre.restype = d
        _lib.oracle_assoc_legendre.argtypes = [i, i, d]
        _lib.oracle_assoc_legendre.restype = d
        _lib.oracle_ylm.argtypes = [i, i, d, d, C.POINTER(d), C.POINTER(d)]
        _lib.oracle_ylm.restype = None
        _lib.oracle_neighbors.argtypes = [i, p, p, i, p, p, p, p, i, C.c_long, p]
        _lib.oracle_neighbors.restype = C.c_long
        _lib.oracle_wigner3j.argtypes = [i] * 6
        _lib.oracle_wigner3j.restype = d
        _lib.oracle_compute.argtypes = [i] * 9 + [p] * 8 + [i, p, p, p, p, i, p, i, i, p, p, p, p, p, p]
        _lib.oracle_compute.restype = i
        _lib.oracle_md.argtypes = [i] * 9 + [p] * 8 + [i, p, p, p, p, p, p, p, i, i, d, p, d, d, p, p, p]
        _lib.oracle_md.restype = i
        _lib.oracle_hnemd_force.argtypes = [i, p, p, p]
        _lib.oracle_hnemd_force.restype = None
        _lib.oracle_heat_current.argtypes = [i, p, p, p, p, p, p]
        _lib.oracle_heat_current.restype = None
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# --- scalar building blocks (Eq. 6-8, Legendre / spherical harmonics) ---------
def fc(r, rc):
    return lib().oracle_fc(float(r), float(rc))


def dfc(r, rc):
    return lib().oracle_dfc(float(r), float(rc))


def fk(k, r, rc):
    return lib().oracle_fk(int(k), float(r), float(rc))


def dfk(k, r, rc):
    return lib().oracle_dfk(int(k), float(r), float(rc))


def chebyshev(k, x):
    return lib().oracle_chebyshev(int(k), float(x))


def dchebyshev(k, x):
    return lib().oracle_dchebyshev(int(k), float(x))


def gn(c, r, rc):
    c = _f64(c)
    return lib().oracle_gn(_ptr(c), c.size, float(r), float(rc))


def dgn(c, r, rc):
    c = _f64(c)
    return lib().oracle_dgn(_ptr(c), c.size, float(r), float(rc))


def legendre(l, x):
    return lib().oracle_legendre(int(l), float(x))


def dlegendre(l, x):
    return lib().oracle_dlegendre(int(l), float(x))


def assoc_legendre(l, m, x):
    return lib().oracle_assoc_legendre(int(l), int(m), float(x))


def wigner3j(j1, j2, j3, m1, m2, m3):
    return lib().oracle_wigner3j(int(j1), int(j2), int(j3), int(m1), int(m2), int(m3))


def ylm(l, m, theta, phi):
    re, im = C.c_double(), C.c_double()
    lib().oracle_ylm(int(l), int(m), float(theta), float(phi), C.byref(re), C.byref(im))
    return complex(re.value, im.value)


# --- neighbours -----------------------------------------------------------------
def neighbors(model, system, use_cells=False):
    """All neighbour pairs as an int array [n_pairs][7]:
    (i, j, sx, sy, sz, in_radial, in_angular), sorted by i, j, shift."""
    L = lib()
    types, pos = _i32(system.types), _f64(system.pos)
    box, pbc = _f64(system.box), _i32(system.pbc)
    rcR, rcA = _f64(model.rc_radial), _f64(model.rc_angular)
    cap = max(1024, system.n * 64)
    while True:
        out = np.empty((cap, 7), np.int32)
        npairs = L.oracle_neighbors(model.n_types, _ptr(rcR), _ptr(rcA), system.n, _ptr(types), _ptr(pos),
                                    _ptr(box), _ptr(pbc), int(use_cells), cap, _ptr(out))
        if npairs == -1:
            raise MemoryError("oracle neighbour build failed")
        if npairs < 0:
            cap = -npairs
            continue
        return out[:npairs].copy()


@dataclass
class OracleResult:
    energy: float
    virial_total: np.ndarray  # [9]
    site_energy: np.ndarray  # [n]
    force: np.ndarray  # [3][n]
    virial: np.ndarray  # [9][n]
    q: np.ndarray | None  # [n][N_des]


def _model_args(m):
    arrs = [_f64(m.rc_radial), _f64(m.rc_angular), _f64(m.c_radial), _f64(m.c_angular),
            _f64(m.w0), _f64(m.b0), _f64(m.w1), _f64(m.b1)]
    ints = [m.n_types, m.n_desc_radial, m.n_desc_angular, m.n_basis_radial, m.n_basis_angular,
            m.l_max, getattr(m, "l_max_4b", 0), getattr(m, "l_max_5b", 0), m.hidden]
    return ints, arrs


def compute(model, system, sample=None, use_cells=None, want_q=False, q_route=0) -> OracleResult:
    """E, F, W (and optionally q) in FP64.  With `sample`, only those beads' U, F,
    W, q are computed (entries of other beads are NaN) and totals are NaN."""
    L = lib()
    n = system.n
    if use_cells is None:
        use_cells = n > 2000
    ints, arrs = _model_args(model)
    types, pos = _i32(system.types), _f64(system.pos)
    box, pbc = _f64(system.box), _i32(system.pbc)
    U = np.full(n, np.nan)
    F = np.full((3, n), np.nan)
    W = np.full((9, n), np.nan)
    q = np.full((n, model.n_des), np.nan) if want_q else None
    e = C.c_double(np.nan)
    wt = np.full(9, np.nan)
    samp = _i32(sample) if sample is not None else None
    rc = L.oracle_compute(*ints, *[_ptr(a) for a in arrs], n, _ptr(types), _ptr(pos), _ptr(box), _ptr(pbc),
                          int(use_cells), _ptr(samp), 0 if samp is None else samp.size, int(q_route),
                          C.byref(e), _ptr(wt), _ptr(U), _ptr(F), _ptr(W), _ptr(q))
    if rc != 0:
        raise RuntimeError(f"oracle_compute failed ({rc})")
    return OracleResult(e.value if sample is None else np.nan, wt, U, F, W, q)


def md(model, system, pos, vel, force, n_steps, dt, use_cells=None, temperature=0.0, tau=1.0, noise=None,
       fe=None):
    """Velocity-Verlet for n_steps (NVE, or NVT with stochastic velocity rescaling
    when noise [n_steps][2] is given; with fe[3] the HNEMD driving force is added
    after every evaluation, and `force` must then include it on entry -- see
    hnemd_force).  pos/vel/force are updated copies.
    Returns (pos, vel, force, thermo[n_steps][2] = (E_pot, E_kin)), plus
    heat[n_steps][6] = (J_pot, J_kin) after each step when fe is given."""
    L = lib()
    n = system.n
    if use_cells is None:
        use_cells = n > 2000
    ints, arrs = _model_args(model)
    types = _i32(system.types)
    pos, vel, force = _f64(pos).copy(), _f64(vel).copy(), _f64(force).copy()
    box, pbc = _f64(system.box), _i32(system.pbc)
    masses = _f64(system.masses)
    thermo = np.zeros((n_steps, 2))
    nz = _f64(noise) if noise is not None else None
    fe_ = _f64(fe) if fe is not None else None
    heat = np.zeros((max(1, n_steps), 6)) if fe is not None else None
    rc = L.oracle_md(*ints, *[_ptr(a) for a in arrs], n, _ptr(types), _ptr(pos), _ptr(vel), _ptr(force),
                     _ptr(masses), _ptr(box), _ptr(pbc), int(use_cells), int(n_steps), float(dt), _ptr(thermo),
                     float(temperature), float(tau), _ptr(nz), _ptr(fe_), _ptr(heat))
    if rc != 0:
        raise RuntimeError("oracle_md failed")
    if fe is not None:
        return pos, vel, force, thermo, heat[:n_steps]
    return pos, vel, force, thermo


def hnemd_force(fe, virial, force):
    """force [3][n] plus the HNEMD driving force of fe[3] from per-particle virials
    virial [9][n] (a new array)."""
    f = _f64(force).copy()
    w = _f64(virial)
    lib().oracle_hnemd_force(f.shape[1], _ptr(_f64(fe)), _ptr(w), _ptr(f))
    return f


def heat_current(system, vel, site_energy, virial):
    """(J_pot[3], J_kin[3]) in eV Angstrom / fs."""
    out = np.zeros(6)
    lib().oracle_heat_current(system.n, _ptr(_i32(system.types)), _ptr(_f64(system.masses)), _ptr(_f64(vel)),
                              _ptr(_f64(site_energy)), _ptr(_f64(virial)), _ptr(out))
    return out[:3], out[3:]


def wrap(system):
    """Positions wrapped into [0, L) on periodic axes, by the oracle's rule."""
    pos = _f64(system.pos).copy()
    for a in range(3):
        if system.pbc[a]:
            L_ = system.box[a]
            inside = (pos[a] >= 0.0) & (pos[a] < L_)
            w = pos[a] - L_ * np.floor(pos[a] / L_)
            w[(w >= L_) | (w < 0.0)] = 0.0
            pos[a] = np.where(inside, pos[a], w)
    return pos


__all__ = ["cg_map", "fc", "dfc", "fk", "dfk", "chebyshev", "dchebyshev", "gn", "dgn", "legendre", "dlegendre",
           "assoc_legendre", "wigner3j", "ylm", "neighbors", "compute", "md", "hnemd_force",
           "heat_current", "wrap", "OracleResult", "lib"]


def cg_map(group_start, group_atoms, mass, pos, box, pbc, force=None, virial=None):
    """Bead positions [3][n_cg], forces [3][n_cg] (or None), virials [9][n_cg] (or None)
    of CSR atom groups (Eq. 9, 12, 14)."""
    L = lib()
    L.oracle_cg_map.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_int] + [C.c_void_p] * 9
    L.oracle_cg_map.restype = None
    st, at = _i32(group_start), _i32(group_atoms)
    n_cg, n_aa = st.size - 1, int(np.asarray(mass).size)
    m, p = _f64(mass), _f64(pos)
    f = _f64(force) if force is not None else None
    w = _f64(virial) if virial is not None else None
    bp = np.zeros((3, n_cg))
    bf = np.zeros((3, n_cg)) if f is not None else None
    bw = np.zeros((9, n_cg)) if w is not None else None
    L.oracle_cg_map(n_cg, _ptr(st), _ptr(at), n_aa, _ptr(m), _ptr(p), _ptr(f), _ptr(w), _ptr(_f64(box)),
                    _ptr(_i32(pbc)), _ptr(bp), _ptr(bf), _ptr(bw))
    return bp, bf, bw
