"""Pins of the oracle's four- and five-body angular descriptors (Sec. II.A, which
refers their definition to the GPUMD paper).  Reading:
    q4_n = sum_{m1 m2 m3} (2 2 2; m1 m2 m3) A_n2m1 A_n2m2 A_n2m3
    q5_n = (q_n1)^2
with A_nlm of Eq. 5 and q_nl of Eq. 4.  They are pinned without the oracle's own
spherical harmonics:
- the Wigner 3j symbols against sympy and their orthogonality relation;
- q4 against kappa tr(Q^3) with the Cartesian tensor Q = sum_j g(r_j)(u_j u_j^T - I/3)
  built in numpy: the cubic rotational invariant of the l = 2 moments is unique up to
  a factor, and one neighbour on the z axis fixes kappa by hand
  (A_2m = g sqrt(5/4pi) delta_m0, tr(Q^3) = 2 g^3 / 9);
- q5 against ((3/4pi) |sum_j g(r_j) u_j|^2)^2 (the l = 1 addition theorem);
- forces against central differences, invariances and the virial identity with both
  terms switched on.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_01234_gb300 import inputs
from tests.test_oracle_system import fd_forces, make_system, np_g, random_rotation

W222 = -math.sqrt(2.0 / 35.0)  # (2 2 2; 0 0 0)
KAPPA = W222 * (5.0 / (4.0 * math.pi)) ** 1.5 * 4.5


def mb_model(T=1, seed=41, l4=2, l5=1, rcR=5.0, rcA=4.0, H=6, nR=3, nA=2, K=5, L=4):
    return inputs.random_model(n_types=T, n_desc_radial=nR, n_desc_angular=nA, n_basis_radial=K,
                               n_basis_angular=K, l_max=L, hidden=H, rc_radial=rcR, rc_angular=rcA,
                               seed=seed, scale=0.3, l_max_4b=l4, l_max_5b=l5)


def cartesian_terms(m, s, i):
    """(q4[n_A], q5[n_A]) of bead i of an open system from Cartesian sums."""
    ti = s.types[i]
    Q = np.zeros((m.n_desc_angular, 3, 3))
    v = np.zeros((m.n_desc_angular, 3))
    for j in range(s.n):
        if j == i:
            continue
        d = s.pos[:, j] - s.pos[:, i]
        r = np.linalg.norm(d)
        tj = s.types[j]
        rc = m.rc_angular[ti, tj]
        if r >= rc:
            continue
        u = d / r
        for n in range(m.n_desc_angular):
            g = np_g(m.c_angular[ti, tj, n], r, rc)
            Q[n] += g * (np.outer(u, u) - np.eye(3) / 3.0)
            v[n] += g * u
    q4 = np.array([KAPPA * np.trace(Q[n] @ Q[n] @ Q[n]) for n in range(m.n_desc_angular)])
    q5 = np.array([(3.0 / (4.0 * math.pi) * v[n] @ v[n]) ** 2 for n in range(m.n_desc_angular)])
    return q4, q5


def test_wigner3j_against_sympy_and_orthogonality():
    wigner = pytest.importorskip("sympy.physics.wigner")
    for args in [(2, 2, 2, 0, 0, 0), (2, 2, 2, 1, -1, 0), (2, 2, 2, 2, -1, -1), (2, 2, 2, -2, 0, 2),
                 (1, 1, 2, 1, 0, -1), (3, 2, 1, -2, 1, 1), (4, 2, 2, 0, 2, -2), (1, 1, 0, 1, -1, 0)]:
        assert oracle.wigner3j(*args) == pytest.approx(float(wigner.wigner_3j(*args)), abs=1e-15), args
    assert oracle.wigner3j(2, 2, 2, 0, 0, 0) == pytest.approx(W222, abs=1e-15)
    assert oracle.wigner3j(2, 2, 2, 1, 1, 0) == 0.0  # m1 + m2 + m3 != 0
    # sum_{m1 m2} (j1 j2 j; m1 m2 m)(j1 j2 j'; m1 m2 m) = delta_jj' / (2j + 1)
    for j, jp in [(2, 2), (3, 3), (2, 4), (1, 3)]:
        m = 0
        s = sum(oracle.wigner3j(2, 2, j, m1, m2, m) * oracle.wigner3j(2, 2, jp, m1, m2, m)
                for m1 in range(-2, 3) for m2 in range(-2, 3))
        assert s == pytest.approx(1.0 / (2 * j + 1) if j == jp else 0.0, abs=1e-14)


def test_descriptor_layout_and_three_body_part_unchanged():
    base = mb_model(l4=0, l5=0, seed=42)
    s = inputs.random_cluster(12, seed=43, box_len=7.0, min_dist=1.3)
    q0 = oracle.compute(base, s, want_q=True).q
    D0 = base.n_des
    nA = base.n_desc_angular
    for l4, l5 in [(2, 0), (0, 1), (2, 1)]:
        m = mb_model(l4=l4, l5=l5, seed=42)
        assert m.n_des == D0 + nA * ((l4 > 0) + (l5 > 0))
        q = oracle.compute(m, s, want_q=True).q
        np.testing.assert_array_equal(q[:, :D0], q0)
        for i in range(s.n):
            c4, c5 = cartesian_terms(m, s, i)
            k = D0
            if l4:
                np.testing.assert_allclose(q[i, k:k + nA], c4, rtol=1e-11, atol=1e-14)
                k += nA
            if l5:
                np.testing.assert_allclose(q[i, k:k + nA], c5, rtol=1e-11, atol=1e-14)
                # five-body = square of the l = 1 three-body descriptor
                np.testing.assert_allclose(q[i, k:k + nA], q0[i, base.n_desc_radial:base.n_desc_radial + nA] ** 2,
                                           rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("r", [1.5, 2.7, 3.6])
def test_single_neighbour_closed_form(r):
    m = mb_model(T=2, seed=44)
    u = np.array([0.3, -0.5, 0.81])
    u /= np.linalg.norm(u)
    s = make_system([[10.0, 10.0, 10.0], list(np.array([10.0, 10.0, 10.0]) + r * u)], [0, 1])
    q = oracle.compute(m, s, want_q=True).q
    D3 = m.n_desc_radial + m.n_desc_angular * m.l_max
    for i, (ti, tj) in enumerate([(0, 1), (1, 0)]):
        for n in range(m.n_desc_angular):
            g = np_g(m.c_angular[ti, tj, n], r, m.rc_angular[ti, tj])
            assert q[i, D3 + n] == pytest.approx(W222 * (5.0 / (4.0 * math.pi)) ** 1.5 * g ** 3, abs=1e-14)
            assert q[i, D3 + m.n_desc_angular + n] == pytest.approx((3.0 / (4.0 * math.pi) * g * g) ** 2, abs=1e-14)


def test_four_body_needs_three_neighbours():
    """Two neighbours at right angles: tr(Q^3) of two orthogonal rank-one tensors is
    (g1^3 + g2^3) 2/9 - (g1^2 g2 + g1 g2^2) / 3, so q4 is not a sum of pair terms."""
    m = mb_model(seed=45, l5=0)
    c = np.array([10.0, 10.0, 10.0])
    r1, r2 = 2.0, 3.1
    s = make_system([c, c + [r1, 0, 0], c + [0, r2, 0]], [0, 0, 0])
    q = oracle.compute(m, s, want_q=True).q
    D3 = m.n_desc_radial + m.n_desc_angular * m.l_max
    for n in range(m.n_desc_angular):
        g1, g2 = (np_g(m.c_angular[0, 0, n], r, 4.0) for r in (r1, r2))
        tr = (g1 ** 3 + g2 ** 3) * 2.0 / 9.0 - (g1 ** 2 * g2 + g1 * g2 ** 2) / 3.0
        assert q[0, D3 + n] == pytest.approx(KAPPA * tr, abs=1e-14)


@pytest.mark.parametrize("l4,l5", [(2, 1), (2, 0), (0, 1)])
def test_forces_fd_open_cluster(l4, l5):
    m = mb_model(T=2, seed=46, l4=l4, l5=l5)
    s = inputs.random_cluster(12, seed=47, box_len=6.5, min_dist=1.2, n_types=2)
    r = oracle.compute(m, s)
    F = fd_forces(m, s)
    scale = np.abs(r.force).max()
    assert np.abs(F - r.force).max() <= 1e-7 * scale + 1e-10
    assert np.abs(r.force.sum(axis=1)).max() < 1e-12 * scale * s.n


def test_forces_fd_small_periodic_images():
    m = mb_model(seed=48)
    s = inputs.random_periodic(6, [6.0, 7.0, 6.5], seed=49, min_dist=1.5)
    r = oracle.compute(m, s)
    F = fd_forces(m, s)
    assert np.abs(F - r.force).max() <= 1e-7 * np.abs(r.force).max() + 1e-10


def test_rotation_invariance_and_virial_identity():
    m = mb_model(T=2, seed=50)
    s = inputs.random_cluster(16, seed=51, box_len=8.0, min_dist=1.1, n_types=2)
    R = random_rotation(52)
    c = s.pos.mean(axis=1, keepdims=True)
    s2 = inputs.System(pos=R @ (s.pos - c) + c, types=s.types, box=s.box, pbc=s.pbc)
    r, r2 = oracle.compute(m, s), oracle.compute(m, s2)
    np.testing.assert_allclose(r2.site_energy, r.site_energy, atol=1e-12)
    np.testing.assert_allclose(r2.force, R @ r.force, atol=1e-12)
    rF = np.einsum("ai,bi->ab", s.pos, r.force).reshape(9)
    np.testing.assert_allclose(r.virial_total, rF, atol=1e-11)


def test_zero_many_body_weights_give_the_three_body_model():
    base = mb_model(T=2, seed=53, l4=0, l5=0)
    m = inputs.ModelParams(**{k: getattr(base, k) for k in base.__dataclass_fields__})
    m.l_max_4b, m.l_max_5b = 2, 1
    m.w0 = np.concatenate([base.w0, np.zeros((2, base.hidden, m.n_des - base.n_des))], axis=2)
    s = inputs.random_cluster(14, seed=54, box_len=7.0, min_dist=1.2, n_types=2)
    a, b = oracle.compute(base, s), oracle.compute(m, s)
    assert a.energy == b.energy
    np.testing.assert_array_equal(a.force, b.force)
    np.testing.assert_array_equal(a.virial, b.virial)
