"""Property-based pins of the oracle's descriptors (Eq. 3-5 and the four- and
five-body terms) over random small clusters drawn by hypothesis:

- every descriptor of every bead is invariant under a rotation or reflection of the
  cluster (O(3): Eq. 4 and the 3j-coupled cube are scalars of the moments) and under
  a relabelling of the beads;
- the four-body term equals kappa tr(Q^3) and the five-body term ((3/4pi)|v|^2)^2,
  both built in numpy from the neighbour vectors, for any geometry;
- q_nl >= 0 (a sum of squared moduli) and the Legendre route equals the Y_lm route.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_01234_gb300 import inputs
from tests.test_oracle_manybody import cartesian_terms, mb_model

hypothesis = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
from hypothesis import given, settings  # noqa: E402

MODEL = mb_model(T=2, seed=60, rcR=5.0, rcA=4.0)


def cluster_from(seed, n):
    s = inputs.random_cluster(n, seed=seed, box_len=6.0, min_dist=1.2, n_types=2)
    s.pos = s.pos + 10.0
    return s


def orthogonal(seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).standard_normal((3, 3)))
    return q * np.sign(np.diag(r))  # any element of O(3), reflections included


@settings(max_examples=25, deadline=None)
@given(seed=st.integers(0, 10**6), n=st.integers(2, 12), rot=st.integers(0, 10**6))
def test_descriptors_invariant_under_o3_and_relabelling(seed, n, rot):
    s = cluster_from(seed, n)
    q = oracle.compute(MODEL, s, want_q=True).q
    R = orthogonal(rot)
    c = s.pos.mean(axis=1, keepdims=True)
    perm = np.random.default_rng(rot + 1).permutation(n)
    s2 = inputs.System(pos=(R @ (s.pos - c) + c)[:, perm].copy(), types=s.types[perm].copy(), box=s.box,
                       pbc=s.pbc)
    q2 = oracle.compute(MODEL, s2, want_q=True).q
    scale = 1e-12 * (1.0 + np.abs(q).max())
    np.testing.assert_allclose(q2, q[perm], rtol=0, atol=scale)


@settings(max_examples=25, deadline=None)
@given(seed=st.integers(0, 10**6), n=st.integers(2, 10))
def test_many_body_terms_equal_their_cartesian_forms(seed, n):
    s = cluster_from(seed, n)
    r = oracle.compute(MODEL, s, want_q=True, q_route=1)
    q0 = oracle.compute(MODEL, s, want_q=True).q
    D3 = MODEL.n_desc_radial + MODEL.n_desc_angular * MODEL.l_max
    nA = MODEL.n_desc_angular
    # the Legendre double sum equals the Y_lm route, and q_nl >= 0
    np.testing.assert_allclose(r.q[:, :D3], q0[:, :D3], rtol=1e-12, atol=1e-14)
    assert np.all(q0[:, MODEL.n_desc_radial:D3] >= -1e-15)
    for i in range(n):
        c4, c5 = cartesian_terms(MODEL, s, i)
        np.testing.assert_allclose(q0[i, D3:D3 + nA], c4, rtol=1e-10, atol=1e-14)
        np.testing.assert_allclose(q0[i, D3 + nA:D3 + 2 * nA], c5, rtol=1e-10, atol=1e-14)
        # the five-body term is the square of the l = 1 three-body term
        np.testing.assert_allclose(q0[i, D3 + nA:], q0[i, MODEL.n_desc_radial:MODEL.n_desc_radial + nA] ** 2,
                                   rtol=1e-12, atol=1e-15)


def test_kappa_value():
    """kappa = (2 2 2; 0 0 0) (5 / 4 pi)^(3/2) 9/2, i.e. -32 sqrt(14) pi^(3/2) / 525 times
    (8 pi / 15)^-3 (the constant of the real-basis form q4 = k tr(M^3), M = 15/(8 pi) Q)."""
    kappa = -math.sqrt(2.0 / 35.0) * (5.0 / (4.0 * math.pi)) ** 1.5 * 4.5
    closed = -32.0 * math.sqrt(14.0) * math.pi ** 1.5 / 525.0 / (8.0 * math.pi / 15.0) ** 3
    assert kappa == pytest.approx(closed, rel=1e-14)
