"""Seeded synthetic inputs: particle configurations, model parameters, velocities.

This module holds no arithmetic of the potential itself (no descriptors, network,
forces or virials).  It only places particles, draws random parameters and draws
velocities, so that the CUDA library and the FP64 oracle can be fed identical
inputs.  Every generator takes an explicit seed and uses numpy's PCG64.

Shapes follow the systems of the paper's Results section (Sec. III): one-bead CG
water (Sec. III.A), a two-type-or-more fullerene-like monolayer (Sec. III.B) and a
mixed atom-and-bead gold nanowire (Sec. III.C).  The paper's trained models and
trajectories are not available, so random-weight models stand in for them.

Units: Angstrom, eV, amu, fs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Boltzmann constant in eV/K and 1 eV/(Angstrom*amu) in Angstrom/fs^2.
KB_EV = 8.617333262e-5
ACC_EV_A_AMU = 9.648533212e-3


@dataclass
class System:
    """One configuration.  pos is SoA [3][n] float64, types int32 [n]."""

    pos: np.ndarray
    types: np.ndarray
    box: np.ndarray  # [3] float64 box lengths (orthorhombic)
    pbc: np.ndarray  # [3] int32, 1 = periodic
    name: str = ""
    vel: np.ndarray | None = None  # SoA [3][n] float64, Angstrom/fs
    masses: np.ndarray | None = None  # per type, amu
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.types.shape[0])


@dataclass
class ModelParams:
    """Hyper-parameters and parameters of one NEP model (Eq. 2, Eq. 6).

    Layouts (row-major):
      rc_radial, rc_angular   [T][T]             cutoff of the pair (t_i, t_j)
      c_radial                [T][T][n_R][K_R]   c^{t_i t_j}_{nk} of the radial g_n
      c_angular               [T][T][n_A][K_A]   same for the angular g_n
      w0                      [T][H][N_des]      hidden-layer weights
      b0                      [T][H]             hidden-layer biases
      w1                      [T][H]             output weights
      b1                      [T]                output bias
    with n_R = n_max^R + 1, K_R = N_bas^R + 1, and
    N_des = n_R + n_A * (l_max + [l_max_4b = 2] + [l_max_5b = 1]): the four-body
    descriptors q4_n (l = 2) follow the three-body ones, then the five-body q5_n
    (l = 1); l_max_4b is 0 or 2, l_max_5b 0 or 1.
    """

    n_types: int
    n_desc_radial: int
    n_desc_angular: int
    n_basis_radial: int
    n_basis_angular: int
    l_max: int
    hidden: int
    rc_radial: np.ndarray
    rc_angular: np.ndarray
    c_radial: np.ndarray
    c_angular: np.ndarray
    w0: np.ndarray
    b0: np.ndarray
    w1: np.ndarray
    b1: np.ndarray
    l_max_4b: int = 0
    l_max_5b: int = 0

    @property
    def n_des(self) -> int:
        return n_descriptors(self.n_desc_radial, self.n_desc_angular, self.l_max, self.l_max_4b, self.l_max_5b)


def n_descriptors(n_desc_radial, n_desc_angular, l_max, l_max_4b=0, l_max_5b=0) -> int:
    return n_desc_radial + n_desc_angular * (l_max + (l_max_4b > 0) + (l_max_5b > 0))


def pair_table(n_types: int, per_type, mix: str = "mean") -> np.ndarray:
    """[T][T] cutoff table; mixed pairs take the arithmetic mean (Sec. III.C)."""
    per_type = np.broadcast_to(np.asarray(per_type, dtype=np.float64), (n_types,))
    t = np.empty((n_types, n_types))
    for a in range(n_types):
        for b in range(n_types):
            t[a, b] = 0.5 * (per_type[a] + per_type[b]) if mix == "mean" else per_type[a]
    return t


def random_model(n_types=1, n_desc_radial=5, n_desc_angular=4, n_basis_radial=8,
                 n_basis_angular=8, l_max=4, hidden=30, rc_radial=8.0, rc_angular=5.0,
                 seed=0, scale=0.1, l_max_4b=0, l_max_5b=0) -> ModelParams:
    """Random-weight model: every parameter ~ N(0, scale^2), drawn in the order
    c_radial, c_angular, w0, b0, w1, b1.  rc_* are scalars (uniform table) or
    [T][T] tables."""
    rng = np.random.default_rng(seed)
    T = n_types
    n_des = n_descriptors(n_desc_radial, n_desc_angular, l_max, l_max_4b, l_max_5b)

    def table(v):
        v = np.asarray(v, dtype=np.float64)
        return np.full((T, T), float(v)) if v.ndim == 0 else v.reshape(T, T).copy()

    cR = scale * rng.standard_normal((T, T, n_desc_radial, n_basis_radial))
    cA = scale * rng.standard_normal((T, T, n_desc_angular, n_basis_angular))
    w0 = scale * rng.standard_normal((T, hidden, n_des))
    b0 = scale * rng.standard_normal((T, hidden))
    w1 = scale * rng.standard_normal((T, hidden))
    b1 = scale * rng.standard_normal((T,))
    return ModelParams(T, n_desc_radial, n_desc_angular, n_basis_radial, n_basis_angular,
                       l_max, hidden, table(rc_radial), table(rc_angular), cR, cA, w0, b0, w1, b1,
                       l_max_4b, l_max_5b)


# ----------------------------------------------------------------------------
# configurations
# ----------------------------------------------------------------------------

def jittered_cubic(n: int, box_len: float, seed: int, min_dist: float = 2.5,
                   jitter: float | None = None) -> System:
    """n beads on a jittered simple-cubic lattice filling a periodic cube.

    m = ceil(n^(1/3)) sites per side; n of the m^3 sites are chosen at random;
    every coordinate gets uniform jitter +-j with j = (spacing - min_dist)/2, which
    keeps every pair at least min_dist apart.
    """
    rng = np.random.default_rng(seed)
    m = int(math.ceil(round(n ** (1.0 / 3.0), 9)))
    while m ** 3 < n:
        m += 1
    a = box_len / m
    if jitter is None:
        jitter = max(0.0, 0.5 * (a - min_dist))
    g = np.arange(m, dtype=np.float64)
    sites = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=0).reshape(3, -1)
    if m ** 3 > n:
        keep = np.sort(rng.choice(m ** 3, size=n, replace=False))
        sites = sites[:, keep]
    pos = (sites + 0.5) * a + rng.uniform(-jitter, jitter, size=sites.shape)
    return System(pos=np.ascontiguousarray(pos), types=np.zeros(n, np.int32),
                  box=np.array([box_len] * 3), pbc=np.ones(3, np.int32),
                  meta={"spacing": a, "jitter": jitter})


def water_small(seed: int = 1000) -> System:
    """512 beads, 8^3 simple cubic at 3.1 A in a 24.8 A periodic cube, +-0.3 A
    uniform jitter (minimum pair distance >= 2.5 A)."""
    s = jittered_cubic(512, 24.8, seed)
    s.name = "water512"
    s.masses = np.array([18.0])
    return s


def water_box(n: int = 100_000, density: float = 0.0334, seed: int = 1001) -> System:
    """One-bead CG water at number density `density` (A^-3) in a periodic cube."""
    L = (n / density) ** (1.0 / 3.0)
    s = jittered_cubic(n, L, seed)
    s.name = f"water{n}"
    s.masses = np.array([18.0])
    return s


def monolayer(nx: int = 250, ny: int = 200, seed: int = 1002, spacing: float = 10.0,
              stretch_y: float = 1.05, sigma: float = 0.2, vacuum: float = 30.0) -> System:
    """Four-type distorted hexagonal monolayer, periodic in x and y, open in z.

    Rectangular cell a x b with a = 2*spacing, b = spacing*sqrt(3)*stretch_y and
    four beads at (0,0), (a/2,0), (a/4,b/2), (3a/4,b/2) of types 0..3; Gaussian
    jitter sigma in x, y and z; the plane sits at z = vacuum/2 in a box of height
    `vacuum`.
    """
    rng = np.random.default_rng(seed)
    a = 2.0 * spacing
    b = spacing * math.sqrt(3.0) * stretch_y
    basis = np.array([[0.0, 0.0], [a / 2, 0.0], [a / 4, b / 2], [3 * a / 4, b / 2]])
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    ox = (ix.reshape(-1, 1) * a + basis[None, :, 0]).reshape(-1)
    oy = (iy.reshape(-1, 1) * b + basis[None, :, 1]).reshape(-1)
    n = ox.size
    types = np.tile(np.arange(4, dtype=np.int32), nx * ny)
    pos = np.stack([ox + 0.25 * spacing, oy + 0.25 * spacing, np.full(n, vacuum / 2)])
    pos = pos + sigma * rng.standard_normal(pos.shape)
    s = System(pos=np.ascontiguousarray(pos), types=types,
               box=np.array([a * nx, b * ny, vacuum]), pbc=np.array([1, 1, 0], np.int32),
               name=f"monolayer{n}", masses=np.full(4, 720.0))
    return s


def nanowire(n_total: int = 1_000_000, seed: int = 1003, a: float = 4.08, n_cells_x: int = 196,
             r_core: float = 15.0, r_inner_sheath: float = 30.0, margin: float = 20.0) -> System:
    """Mixed atom-and-bead wire along x (periodic in x, open in y and z).

    The cross-section is tiled by cubic cells of side `a`.  Cells whose centre lies
    within r_core of the axis hold the 4 atoms of an FCC cell (type 0); every other
    cell holds one bead at its centre, type 1 within r_inner_sheath and type 2
    beyond.  Bead sites are taken in order of distance from the axis until the
    total reaches n_total.  A tiny seeded jitter (0.05 A) breaks lattice symmetry.
    """
    rng = np.random.default_rng(seed)
    Lx = n_cells_x * a
    # cross-section cells large enough for n_total
    r_guess = math.sqrt(n_total / n_cells_x * a * a / math.pi) + 4 * a
    m = int(math.ceil(2 * r_guess / a)) + 2
    c = (np.arange(m) - (m - 1) / 2.0) * a
    cy, cz = np.meshgrid(c, c, indexing="ij")
    cy, cz = cy.reshape(-1), cz.reshape(-1)
    rho = np.hypot(cy, cz)
    order = np.lexsort((cz, cy, rho))
    cy, cz, rho = cy[order], cz[order], rho[order]
    core = rho <= r_core
    fcc = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]]) * a
    xs = np.arange(n_cells_x) * a
    # atoms: cell corner at (x, cy - a/2, cz - a/2)
    ay = np.concatenate([cy[core] - a / 2 + f[1] for f in fcc])
    az = np.concatenate([cz[core] - a / 2 + f[2] for f in fcc])
    afx = np.concatenate([np.full(core.sum(), f[0]) for f in fcc])
    atom_x = (xs[:, None] + afx[None, :]).reshape(-1)
    atom_y = np.tile(ay, n_cells_x)
    atom_z = np.tile(az, n_cells_x)
    n_atoms = atom_x.size
    n_beads = n_total - n_atoms
    sy, sz, srho = cy[~core], cz[~core], rho[~core]
    # bead sites ordered by rho, then by x layer
    n_cells_needed = int(math.ceil(n_beads / n_cells_x))
    sy, sz, srho = sy[:n_cells_needed], sz[:n_cells_needed], srho[:n_cells_needed]
    bx = np.repeat((xs + a / 2)[None, :], sy.size, axis=0).reshape(-1)
    by = np.repeat(sy, n_cells_x)
    bz = np.repeat(sz, n_cells_x)
    brho = np.repeat(srho, n_cells_x)
    bx, by, bz, brho = bx[:n_beads], by[:n_beads], bz[:n_beads], brho[:n_beads]
    btype = np.where(brho <= r_inner_sheath, 1, 2).astype(np.int32)
    r_out = float(brho.max()) if n_beads else r_core
    side = 2 * (r_out + a) + 2 * margin
    pos = np.stack([np.concatenate([atom_x, bx]), np.concatenate([atom_y, by]) + side / 2,
                    np.concatenate([atom_z, bz]) + side / 2])
    pos = pos + 0.05 * rng.standard_normal(pos.shape)
    types = np.concatenate([np.zeros(n_atoms, np.int32), btype])
    return System(pos=np.ascontiguousarray(pos), types=types, box=np.array([Lx, side, side]),
                  pbc=np.array([1, 0, 0], np.int32), name=f"nanowire{n_total}",
                  masses=np.array([196.97, 4 * 196.97, 4 * 196.97]),
                  meta={"n_atoms": n_atoms, "r_out": r_out})


def maxwell_boltzmann(system: System, temperature: float, seed: int) -> np.ndarray:
    """SoA [3][n] velocities (A/fs) at `temperature`, zero total momentum, rescaled
    so that 2*KE/((3n-3)*kB) equals `temperature` exactly."""
    rng = np.random.default_rng(seed)
    m = system.masses[system.types]
    sigma = np.sqrt(KB_EV * temperature / m * ACC_EV_A_AMU)
    v = rng.standard_normal((3, system.n)) * sigma[None, :]
    p = (v * m[None, :]).sum(axis=1) / m.sum()
    v -= p[:, None]
    ke = 0.5 * (m[None, :] * v * v).sum() / ACC_EV_A_AMU
    t_now = 2.0 * ke / ((3 * system.n - 3) * KB_EV)
    v *= math.sqrt(temperature / t_now)
    return np.ascontiguousarray(v)


def random_cluster(n: int, seed: int, box_len: float = 12.0, min_dist: float = 1.0,
                   n_types: int = 1) -> System:
    """Small open cluster (no periodicity) with random positions, for invariance
    and finite-difference checks.  Rejection sampling enforces min_dist."""
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < n:
        p = rng.uniform(0.0, box_len, size=3)
        if all(np.linalg.norm(p - q) >= min_dist for q in pts):
            pts.append(p)
    pos = np.ascontiguousarray(np.array(pts).T)
    types = rng.integers(0, n_types, size=n).astype(np.int32)
    return System(pos=pos, types=types, box=np.array([box_len] * 3),
                  pbc=np.zeros(3, np.int32), name=f"cluster{n}",
                  masses=np.full(n_types, 18.0))


def random_periodic(n: int, box, seed: int, min_dist: float = 1.2, n_types: int = 1,
                    pbc=(1, 1, 1)) -> System:
    """n particles uniformly at random in a box (rejection for min_dist, periodic
    distance on periodic axes)."""
    rng = np.random.default_rng(seed)
    box = np.asarray(box, dtype=np.float64)
    pbc = np.asarray(pbc, dtype=np.int32)
    pts = np.empty((0, 3))
    while pts.shape[0] < n:
        p = rng.uniform(0.0, 1.0, size=3) * box
        if pts.shape[0]:
            d = pts - p
            d = d - pbc * box * np.round(d / box)
            if np.min(np.einsum("ij,ij->i", d, d)) < min_dist ** 2:
                continue
        pts = np.vstack([pts, p])
    types = rng.integers(0, n_types, size=n).astype(np.int32)
    return System(pos=np.ascontiguousarray(pts.T), types=types, box=box, pbc=pbc,
                  name=f"random{n}", masses=np.full(n_types, 18.0))


def request_stream(n_requests: int = 4096, seed: int = 1004, n_min: int = 64,
                   n_max: int = 4096, density: float = 0.0334):
    """Mixed served requests: bead counts log-uniform in [n_min, n_max]; a seeded
    coin picks a water-like cube (model 0) or a four-type monolayer patch (model 1).
    Yields (model_id, System) pairs."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n_requests):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        if rng.uniform() < 0.5:
            L = (n / density) ** (1.0 / 3.0)
            s = jittered_cubic(n, L, seed + 7919 * (r + 1))
            s.name = f"req{r}-water{n}"
            s.masses = np.array([18.0])
            out.append((0, s))
        else:
            cells = max(1, n // 4)
            nx = max(2, int(round(math.sqrt(cells * 18.187 / 20.0))))
            ny = max(2, int(round(cells / nx)))
            s = monolayer(nx, ny, seed=seed + 7919 * (r + 1))
            s.name = f"req{r}-monolayer{s.n}"
            out.append((1, s))
    return out
