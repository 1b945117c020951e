"""Pins of the whole oracle evaluation (Eq. 1-5, 15-16 and F = -grad E) against
closed forms, finite differences, invariances and brute-force neighbour search."""
import math

import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb
from scipy import special

import oracle
from paper_2603_01234_gb300 import inputs


def small_model(T=1, seed=11, rcR=5.0, rcA=4.0, H=6, nR=3, nA=2, K=5, L=4):
    return inputs.random_model(n_types=T, n_desc_radial=nR, n_desc_angular=nA, n_basis_radial=K,
                               n_basis_angular=K, l_max=L, hidden=H, rc_radial=rcR, rc_angular=rcA,
                               seed=seed, scale=0.3)


def np_g(c, r, rc):
    """g_n(r) for a coefficient vector, via numpy's Chebyshev evaluation."""
    x = 2 * (r / rc - 1) ** 2 - 1
    fcut = 0.5 * (1 + math.cos(math.pi * r / rc)) if r < rc else 0.0
    return sum(ck * 0.5 * (npcheb.chebval(x, np.eye(len(c))[k]) + 1) * fcut for k, ck in enumerate(c))


def np_net(m, t, q):
    x = m.w0[t] @ q - m.b0[t]
    return float(m.w1[t] @ np.tanh(x) - m.b1[t])


def make_system(pos, types, box=30.0, pbc=(0, 0, 0)):
    pos = np.asarray(pos, dtype=np.float64).T.copy()
    return inputs.System(pos=pos, types=np.asarray(types, np.int32), box=np.array([box] * 3),
                         pbc=np.array(pbc, np.int32), masses=np.ones(4) * 18.0)


# Eq. 2 special case: w0 = 0 makes U = sum w1 tanh(-b0) - b1 (signs of both biases)
def test_network_bias_signs():
    m = small_model()
    m.w0[:] = 0.0
    m.b0[:] = math.atanh(0.5)
    s = make_system([[10, 10, 10], [12, 10, 10]], [0, 0])
    r = oracle.compute(m, s)
    expect = float(m.w1[0].sum() * -0.5 - m.b1[0])
    assert r.site_energy[0] == pytest.approx(expect, abs=1e-14)
    assert r.energy == pytest.approx(2 * expect, abs=1e-13)
    assert np.abs(r.force).max() < 1e-14


# Two beads: q_n = g_n(r), q_nl = (2l+1)/(4 pi) g_n^A(r)^2; asymmetric c^{t_i t_j}
@pytest.mark.parametrize("r", [1.5, 3.0, 3.9, 4.5])
def test_two_bead_closed_form(r):
    m = small_model(T=2, seed=12)
    s = make_system([[10, 10, 10], [10 + r / math.sqrt(3), 10 + r / math.sqrt(3), 10 + r / math.sqrt(3)]], [0, 1])
    res = oracle.compute(m, s, want_q=True)
    for i, (ti, tj) in enumerate([(0, 1), (1, 0)]):
        q = np.zeros(m.n_des)
        for n in range(m.n_desc_radial):
            q[n] = np_g(m.c_radial[ti, tj, n], r, m.rc_radial[ti, tj])
        for l in range(1, m.l_max + 1):
            for n in range(m.n_desc_angular):
                g = np_g(m.c_angular[ti, tj, n], r, m.rc_angular[ti, tj]) if r < m.rc_angular[ti, tj] else 0.0
                q[m.n_desc_radial + (l - 1) * m.n_desc_angular + n] = (2 * l + 1) / (4 * math.pi) * g * g
        np.testing.assert_allclose(res.q[i], q, atol=1e-13)
        assert res.site_energy[i] == pytest.approx(np_net(m, ti, q), abs=1e-13)
    # the force is along the axis and equals -dE/dr
    h = 1e-5

    def energy_at(rr):
        ss = make_system([[10, 10, 10], [10 + rr / math.sqrt(3)] * 3], [0, 1])
        return oracle.compute(m, ss).energy
    dEdr = (energy_at(r + h) - energy_at(r - h)) / (2 * h)
    u = np.ones(3) / math.sqrt(3)
    np.testing.assert_allclose(res.force[:, 1], -dEdr * u, atol=1e-8)
    np.testing.assert_allclose(res.force[:, 0], dEdr * u, atol=1e-8)


# Three beads: q_nl(i) = (2l+1)/(4pi) [g1^2 + g2^2 + 2 g1 g2 P_l(cos theta)]
@pytest.mark.parametrize("theta", np.linspace(0.3, math.pi, 6))
def test_three_bead_angle_scan(theta):
    m = small_model(seed=13, rcR=6.0, rcA=5.0)
    r1, r2 = 2.2, 3.1
    c = np.array([15.0, 15, 15])
    p1 = c + r1 * np.array([1, 0, 0])
    p2 = c + r2 * np.array([math.cos(theta), math.sin(theta), 0])
    s = make_system([c, p1, p2], [0, 0, 0])
    res = oracle.compute(m, s, want_q=True)
    for l in range(1, 5):
        for n in range(m.n_desc_angular):
            g1 = np_g(m.c_angular[0, 0, n], r1, 5.0)
            g2 = np_g(m.c_angular[0, 0, n], r2, 5.0)
            expect = (2 * l + 1) / (4 * math.pi) * (g1 * g1 + g2 * g2 + 2 * g1 * g2 * special.eval_legendre(l, math.cos(theta)))
            assert res.q[0, m.n_desc_radial + (l - 1) * m.n_desc_angular + n] == pytest.approx(expect, abs=1e-13)


def fd_forces(m, s, h=1e-5, beads=None):
    beads = range(s.n) if beads is None else beads
    F = np.zeros((3, s.n))
    for i in beads:
        for a in range(3):
            sp = inputs.System(pos=s.pos.copy(), types=s.types, box=s.box, pbc=s.pbc)
            sm = inputs.System(pos=s.pos.copy(), types=s.types, box=s.box, pbc=s.pbc)
            sp.pos[a, i] += h
            sm.pos[a, i] -= h
            F[a, i] = -(oracle.compute(m, sp).energy - oracle.compute(m, sm).energy) / (2 * h)
    return F


# F = -grad E by central differences: open two-type cluster
def test_forces_fd_open_cluster():
    m = small_model(T=2, seed=14)
    s = inputs.random_cluster(14, seed=5, box_len=7.0, min_dist=1.2, n_types=2)
    r = oracle.compute(m, s)
    F = fd_forces(m, s)
    scale = np.abs(r.force).max()
    assert np.abs(F - r.force).max() <= 1e-7 * scale + 1e-10


# ... and a periodic box smaller than 2 r_c, where beads see their own images
def test_forces_fd_small_periodic_images():
    m = small_model(seed=15, rcR=5.0, rcA=4.0)
    s = inputs.random_periodic(6, [6.0, 7.0, 6.5], seed=6, min_dist=1.5)
    r = oracle.compute(m, s)
    F = fd_forces(m, s)
    scale = np.abs(r.force).max()
    assert np.abs(F - r.force).max() <= 1e-7 * scale + 1e-10
    assert np.abs(r.force.sum(axis=1)).max() < 1e-12 * scale * s.n


def test_total_force_zero_and_translation():
    m = small_model(T=2, seed=16)
    s = inputs.random_cluster(20, seed=7, box_len=8.0, min_dist=1.1, n_types=2)
    r = oracle.compute(m, s)
    assert np.abs(r.force.sum(axis=1)).max() < 1e-12 * (1 + np.abs(r.force).max()) * s.n
    s2 = inputs.System(pos=s.pos + np.array([[1.7], [-3.2], [0.4]]), types=s.types, box=s.box, pbc=s.pbc)
    r2 = oracle.compute(m, s2)
    assert r2.energy == pytest.approx(r.energy, rel=1e-12)
    np.testing.assert_allclose(r2.force, r.force, atol=1e-12)


def random_rotation(seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((3, 3)))
    return q * np.sign(np.linalg.det(q))


def test_rotation_invariance_and_covariance():
    m = small_model(T=2, seed=17)
    s = inputs.random_cluster(16, seed=8, box_len=8.0, min_dist=1.1, n_types=2)
    R = random_rotation(9)
    c = s.pos.mean(axis=1, keepdims=True)
    s2 = inputs.System(pos=R @ (s.pos - c) + c, types=s.types, box=s.box, pbc=s.pbc)
    r, r2 = oracle.compute(m, s), oracle.compute(m, s2)
    assert r2.energy == pytest.approx(r.energy, rel=1e-12)
    np.testing.assert_allclose(r2.site_energy, r.site_energy, atol=1e-12)
    np.testing.assert_allclose(r2.force, R @ r.force, atol=1e-12)
    # per-bead virial co-rotates: W' = R W R^T
    for i in range(s.n):
        W = r.virial[:, i].reshape(3, 3)
        np.testing.assert_allclose(r2.virial[:, i].reshape(3, 3), R @ W @ R.T, atol=1e-11)


def test_permutation_invariance():
    m = small_model(T=2, seed=18)
    s = inputs.random_cluster(16, seed=10, box_len=8.0, min_dist=1.1, n_types=2)
    perm = np.random.default_rng(3).permutation(s.n)
    s2 = inputs.System(pos=s.pos[:, perm].copy(), types=s.types[perm].copy(), box=s.box, pbc=s.pbc)
    r, r2 = oracle.compute(m, s), oracle.compute(m, s2)
    assert r2.energy == pytest.approx(r.energy, rel=1e-12)
    np.testing.assert_allclose(r2.force, r.force[:, perm], atol=1e-12)
    np.testing.assert_allclose(r2.virial, r.virial[:, perm], atol=1e-12)


# Type information enters only through the parameters (c^{ij}, per-type network):
# a two-type model whose types share all parameters equals the one-type model.
def test_types_only_through_parameters():
    m1 = small_model(T=1, seed=19)
    m2 = small_model(T=2, seed=19)
    for name in ("c_radial", "c_angular"):
        getattr(m2, name)[:] = getattr(m1, name)[0, 0][None, None]
    for name in ("w0", "b0", "w1", "b1"):
        getattr(m2, name)[:] = getattr(m1, name)[0]
    s = inputs.random_cluster(15, seed=11, box_len=8.0, min_dist=1.1, n_types=2)
    s1 = inputs.System(pos=s.pos, types=np.zeros(s.n, np.int32), box=s.box, pbc=s.pbc)
    assert oracle.compute(m2, s).energy == pytest.approx(oracle.compute(m1, s1).energy, rel=1e-13)
    # while distinct c^{01} makes the labels matter
    m2.c_radial[0, 1] += 0.2
    assert abs(oracle.compute(m2, s).energy - oracle.compute(m1, s1).energy) > 1e-6


# Eq. 15-16 for an open cluster: sum_i W_i = sum_i r_i (x) F_i
def test_virial_open_cluster_identity():
    m = small_model(T=2, seed=20)
    s = inputs.random_cluster(18, seed=12, box_len=8.0, min_dist=1.1, n_types=2)
    r = oracle.compute(m, s)
    rF = np.einsum("ai,bi->ab", s.pos, r.force).reshape(9)
    np.testing.assert_allclose(r.virial_total, rF, atol=1e-11)
    np.testing.assert_allclose(r.virial.sum(axis=1), r.virial_total, atol=1e-12)
    Wt = r.virial_total.reshape(3, 3)
    np.testing.assert_allclose(Wt, Wt.T, atol=1e-11)


# periodic: W_aa = -dE/d(eps_aa) under an affine stretch of box and positions
# (an orthorhombic box admits only the diagonal strains)
def test_virial_periodic_strain_derivative():
    m = small_model(seed=21, rcR=5.0, rcA=4.0)
    s = inputs.random_periodic(20, [9.0, 10.0, 11.0], seed=13, min_dist=1.4)
    r = oracle.compute(m, s)
    W = r.virial_total.reshape(3, 3)
    h = 1e-6
    for a in range(3):
        E = []
        for sg in (1, -1):
            scale = np.ones(3)
            scale[a] += sg * h
            st = inputs.System(pos=s.pos * scale[:, None], types=s.types, box=s.box * scale, pbc=s.pbc)
            E.append(oracle.compute(m, st).energy)
        assert -(E[0] - E[1]) / (2 * h) == pytest.approx(W[a, a], rel=1e-6, abs=1e-9)


def test_neighbors_brute_vs_cells_vs_numpy():
    m = small_model(seed=22, rcR=5.0, rcA=3.5)
    s = inputs.random_periodic(300, [16.0, 17.0, 18.0], seed=14, min_dist=1.2)
    nb_b = oracle.neighbors(m, s, use_cells=False)
    nb_c = oracle.neighbors(m, s, use_cells=True)
    np.testing.assert_array_equal(nb_b, nb_c)
    # numpy minimum-image brute force (box > 2 rc on every axis)
    w = oracle.wrap(s)
    d = w[:, None, :] - w[:, :, None]  # d[a, i, j] = x_j - x_i
    sh = -np.round(d / s.box[:, None, None])
    d = d + sh * s.box[:, None, None]
    r2 = (d * d).sum(axis=0)
    np.fill_diagonal(r2, np.inf)
    ii, jj = np.nonzero(r2 < 25.0)
    assert len(ii) == int(nb_b[:, 5].sum())
    got = set(map(tuple, nb_b[nb_b[:, 5] == 1][:, :5]))
    want = set((i, j, *sh[:, i, j].astype(int)) for i, j in zip(ii, jj))
    assert got == want
    ia, ja = np.nonzero(r2 < 3.5 ** 2)
    assert len(ia) == int(nb_b[:, 6].sum())


def test_neighbors_open_axis_cells():
    m = small_model(seed=23, rcR=5.0, rcA=3.5)
    s = inputs.random_periodic(250, [18.0, 18.0, 25.0], seed=15, min_dist=1.2, pbc=(1, 1, 0))
    np.testing.assert_array_equal(oracle.neighbors(m, s, use_cells=False), oracle.neighbors(m, s, use_cells=True))


def test_self_images_counted_in_small_box():
    """L = 4 < r_c = 5: a single bead sees its own periodic images."""
    m = small_model(seed=24, rcR=5.0, rcA=4.5)
    s = inputs.System(pos=np.array([[1.0], [1.0], [1.0]]), types=np.zeros(1, np.int32),
                      box=np.array([4.0, 4.0, 4.0]), pbc=np.ones(3, np.int32))
    nb = oracle.neighbors(m, s)
    # image shifts n with 0 < 4|n| < 5: the 6 face neighbours only
    assert int(nb[:, 5].sum()) == 6 and int(nb[:, 6].sum()) == 6
    r = oracle.compute(m, s)
    assert np.abs(r.force).max() < 1e-13  # a lone bead in a cubic lattice feels no force


# velocity-Verlet: energy fluctuation shrinks ~dt^2 (second order)
def test_md_energy_conservation_second_order():
    m = small_model(seed=25, rcR=5.0, rcA=4.0)
    s = inputs.random_periodic(24, [10.0, 10.0, 10.0], seed=16, min_dist=2.0)
    s.masses = np.array([18.0])
    v = inputs.maxwell_boltzmann(s, 300.0, seed=17)
    f0 = oracle.compute(m, s).force
    spread = []
    for dt in (1.0, 0.5):
        steps = int(round(40 / dt))
        _, _, _, th = oracle.md(m, s, s.pos, v, f0, steps, dt)
        etot = th.sum(axis=1)
        spread.append(etot.max() - etot.min())
    assert spread[1] < spread[0] / 3.0
    assert spread[0] < 1e-2


# Stochastic velocity rescaling: for an ideal gas (no forces) the resampled kinetic
# energy follows the canonical Gamma distribution, mean N_f kT/2, variance N_f (kT)^2/2.
def test_bussi_thermostat_canonical_kinetic_energy():
    m = small_model(seed=26, rcR=2.0, rcA=1.5)
    m.w1[:] = 0.0  # U_i = -b1: no forces
    s = inputs.random_periodic(12, [40.0, 40.0, 40.0], seed=27, min_dist=3.0)
    s.masses = np.array([18.0])
    v = inputs.maxwell_boltzmann(s, 50.0, seed=28)
    steps, T, tau = 30000, 300.0, 50.0
    rng = np.random.default_rng(29)
    nf = 3 * s.n - 3
    noise = np.stack([rng.standard_normal(steps), rng.chisquare(nf - 1, size=steps)], axis=1)
    f0 = np.zeros_like(s.pos)
    _, _, f, th = oracle.md(m, s, s.pos, v, f0, steps, 5.0, temperature=T, tau=tau, noise=noise)
    assert np.abs(f).max() == 0.0
    K = th[2000:, 1]
    kT = inputs.KB_EV * T
    assert K.mean() == pytest.approx(nf * kT / 2, rel=0.05)
    assert K.var() == pytest.approx(nf * kT * kT / 2, rel=0.2)
