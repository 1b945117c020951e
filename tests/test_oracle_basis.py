"""Pins of the oracle's building blocks (Eq. 6-8, Legendre, spherical harmonics)
against closed forms, library routines and quadrature -- not against itself."""
import math

import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb
from numpy.polynomial import legendre as npleg
from scipy import special

import oracle


# Eq. 8: f_c(0) = 1, f_c(rc/2) = 1/2, f_c(rc) = 0, zero beyond, zero slope at rc
@pytest.mark.parametrize("rc", [5.0, 8.0, 15.0])
def test_cutoff_closed_form(rc):
    assert oracle.fc(0.0, rc) == pytest.approx(1.0, abs=1e-15)
    assert oracle.fc(rc / 2, rc) == pytest.approx(0.5, abs=1e-15)
    assert oracle.fc(rc, rc) == pytest.approx(0.0, abs=1e-15)
    assert oracle.fc(rc * 1.01, rc) == 0.0
    assert oracle.dfc(rc, rc) == pytest.approx(0.0, abs=1e-15)
    assert oracle.dfc(rc / 2, rc) == pytest.approx(-0.5 * math.pi / rc, rel=1e-14)
    for r in np.linspace(0.3, rc - 0.3, 7):
        h = 1e-6
        fd = (oracle.fc(r + h, rc) - oracle.fc(r - h, rc)) / (2 * h)
        assert oracle.dfc(r, rc) == pytest.approx(fd, rel=1e-7, abs=1e-10)


# Chebyshev T_k and T_k' against numpy's polynomial module
def test_chebyshev_vs_numpy():
    xs = np.linspace(-1.0, 1.0, 41)
    for k in range(12):
        c = np.zeros(k + 1)
        c[k] = 1.0
        dc = npcheb.chebder(c)
        for x in xs:
            assert oracle.chebyshev(k, x) == pytest.approx(npcheb.chebval(x, c), abs=1e-12)
            assert oracle.dchebyshev(k, x) == pytest.approx(npcheb.chebval(x, dc), abs=1e-9 * max(1, k * k))


# Eq. 7: f_0 = f_c and f_1 = (r/rc - 1)^2 f_c; derivative = central FD
def test_fk_closed_forms_and_derivative():
    rc = 8.0
    for r in np.linspace(0.1, 7.9, 25):
        assert oracle.fk(0, r, rc) == pytest.approx(oracle.fc(r, rc), abs=1e-15)
        assert oracle.fk(1, r, rc) == pytest.approx((r / rc - 1) ** 2 * oracle.fc(r, rc), abs=1e-14)
        for k in range(9):
            h = 1e-6
            fd = (oracle.fk(k, r + h, rc) - oracle.fk(k, r - h, rc)) / (2 * h)
            assert oracle.dfk(k, r, rc) == pytest.approx(fd, abs=2e-8)
    # beyond the cutoff every basis function vanishes
    assert all(oracle.fk(k, 8.5, rc) == 0.0 for k in range(9))


# Eq. 6 is a plain linear combination
def test_gn_is_linear_combination():
    rng = np.random.default_rng(3)
    c = rng.standard_normal(8)
    rc = 5.0
    for r in (0.7, 2.0, 4.9):
        assert oracle.gn(c, r, rc) == pytest.approx(sum(c[k] * oracle.fk(k, r, rc) for k in range(8)), abs=1e-14)


# Legendre P_l, P_l' and associated P_l^m against scipy / numpy
def test_legendre_vs_library():
    for l in range(7):
        c = np.zeros(l + 1)
        c[l] = 1.0
        for x in np.linspace(-1, 1, 21):
            assert oracle.legendre(l, x) == pytest.approx(special.eval_legendre(l, x), abs=1e-13)
            assert oracle.dlegendre(l, x) == pytest.approx(npleg.legval(x, npleg.legder(c)), abs=1e-11)
        for m in range(l + 1):
            for x in np.linspace(-0.99, 0.99, 9):
                assert oracle.assoc_legendre(l, m, x) == pytest.approx(special.lpmv(m, l, x), rel=1e-11, abs=1e-12)


# complex Y_lm against scipy's sph_harm_y (theta polar, phi azimuth)
def test_ylm_vs_scipy():
    rng = np.random.default_rng(4)
    for _ in range(20):
        th, ph = rng.uniform(0, math.pi), rng.uniform(-math.pi, math.pi)
        for l in range(5):
            for m in range(-l, l + 1):
                ref = complex(special.sph_harm_y(l, m, th, ph))
                got = oracle.ylm(l, m, th, ph)
                assert abs(got - ref) < 1e-12


# orthonormality by Gauss-Legendre (cos theta) x uniform (phi) quadrature
def test_ylm_orthonormal_quadrature():
    xg, wg = npleg.leggauss(16)
    nphi = 24
    phis = 2 * math.pi * np.arange(nphi) / nphi
    lm = [(l, m) for l in range(1, 5) for m in range(-l, l + 1)]
    Y = np.array([[oracle.ylm(l, m, math.acos(x), p) for x in xg for p in phis] for (l, m) in lm])
    w = np.repeat(wg, nphi) * (2 * math.pi / nphi)
    G = (Y * w[None, :]) @ Y.conj().T
    assert np.abs(G - np.eye(len(lm))).max() < 1e-12


# addition theorem: sum_m Y_lm(u) conj Y_lm(v) = (2l+1)/(4 pi) P_l(u.v)
def test_addition_theorem():
    rng = np.random.default_rng(5)
    for _ in range(10):
        a = rng.standard_normal(3)
        b = rng.standard_normal(3)
        a /= np.linalg.norm(a)
        b /= np.linalg.norm(b)
        ta, pa = math.acos(a[2]), math.atan2(a[1], a[0])
        tb, pb = math.acos(b[2]), math.atan2(b[1], b[0])
        for l in range(1, 5):
            s = sum(oracle.ylm(l, m, ta, pa) * oracle.ylm(l, m, tb, pb).conjugate() for m in range(-l, l + 1))
            assert s.real == pytest.approx((2 * l + 1) / (4 * math.pi) * special.eval_legendre(l, a @ b), abs=1e-13)
            assert abs(s.imag) < 1e-13
