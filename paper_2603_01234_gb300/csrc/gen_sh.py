"""Generate sh_poly.cuh: real orthonormal spherical harmonics l = 1..4 as homogeneous
harmonic polynomials of the unit vector (the angular moments of Eq. 5), and the
harmonics' sphere-reduced form (z^2 = 1 - x^2 - y^2) from which the angular pair
forces are evaluated.

Run with sympy available:  python gen_sh.py > sh_poly.cuh
The script checks harmonicity, homogeneity and orthonormality before writing.
"""
import sys

import numpy as np
import sympy as sp
from numpy.polynomial import legendre as npleg

x, y, z = sp.symbols("x y z", real=True)
r2 = x * x + y * y + z * z
pi = sp.pi
S = sp.sqrt
Q = sp.Rational

# (l, m) -> homogeneous harmonic polynomial of degree l, normalised on the unit sphere
Y = {
    (1, -1): S(3 / (4 * pi)) * y, (1, 0): S(3 / (4 * pi)) * z, (1, 1): S(3 / (4 * pi)) * x,
    (2, -2): S(15 / pi) / 2 * x * y, (2, -1): S(15 / pi) / 2 * y * z,
    (2, 0): S(5 / pi) / 4 * (2 * z * z - x * x - y * y),
    (2, 1): S(15 / pi) / 2 * x * z, (2, 2): S(15 / pi) / 4 * (x * x - y * y),
    (3, -3): S(35 / (2 * pi)) / 4 * y * (3 * x * x - y * y), (3, -2): S(105 / pi) / 2 * x * y * z,
    (3, -1): S(21 / (2 * pi)) / 4 * y * (4 * z * z - x * x - y * y),
    (3, 0): S(7 / pi) / 4 * z * (2 * z * z - 3 * x * x - 3 * y * y),
    (3, 1): S(21 / (2 * pi)) / 4 * x * (4 * z * z - x * x - y * y),
    (3, 2): S(105 / pi) / 4 * z * (x * x - y * y), (3, 3): S(35 / (2 * pi)) / 4 * x * (x * x - 3 * y * y),
    (4, -4): Q(3, 4) * S(35 / pi) * x * y * (x * x - y * y),
    (4, -3): Q(3, 4) * S(35 / (2 * pi)) * y * z * (3 * x * x - y * y),
    (4, -2): Q(3, 4) * S(5 / pi) * x * y * (6 * z * z - x * x - y * y),
    (4, -1): Q(3, 4) * S(5 / (2 * pi)) * y * z * (4 * z * z - 3 * x * x - 3 * y * y),
    (4, 0): Q(3, 16) * S(1 / pi) * (35 * z ** 4 - 30 * z * z * r2 + 3 * r2 * r2),
    (4, 1): Q(3, 4) * S(5 / (2 * pi)) * x * z * (4 * z * z - 3 * x * x - 3 * y * y),
    (4, 2): Q(3, 8) * S(5 / pi) * (x * x - y * y) * (6 * z * z - x * x - y * y),
    (4, 3): Q(3, 4) * S(35 / (2 * pi)) * x * z * (x * x - 3 * y * y),
    (4, 4): Q(3, 16) * S(35 / pi) * (x * x * (x * x - 3 * y * y) - y * y * (3 * x * x - y * y)),
}
KEYS = [(l, m) for l in range(1, 5) for m in range(-l, l + 1)]


def check():
    for k in KEYS:
        v = Y[k]
        assert sp.simplify(sp.diff(v, x, 2) + sp.diff(v, y, 2) + sp.diff(v, z, 2)) == 0
        p = sp.Poly(sp.expand(v), x, y, z)
        assert p.is_homogeneous and p.total_degree() == k[0]
    xg, wg = npleg.leggauss(20)
    nphi = 40
    ph = 2 * np.pi * np.arange(nphi) / nphi
    ct = np.repeat(xg, nphi)
    st = np.sqrt(1 - ct ** 2)
    pp = np.tile(ph, len(xg))
    X, Yv, Z = st * np.cos(pp), st * np.sin(pp), ct
    w = np.repeat(wg, nphi) * 2 * np.pi / nphi
    M = np.array([sp.lambdify((x, y, z), Y[k], "numpy")(X, Yv, Z) * np.ones_like(X) for k in KEYS])
    assert np.abs((M * w) @ M.T - np.eye(len(KEYS))).max() < 1e-12


def c(expr):
    e = sp.expand(sp.N(expr, 20))
    s = sp.ccode(e)
    # numeric literals -> real(...) so that float kernels stay in float
    import re
    s = re.sub(r"(\d+\.\d+(e[-+]?\d+)?)", r"real(\1)", s)
    return re.sub(r"pow\(([xyz]), (\d)\)", r"\1\2", s)


MONO = ("    const real x2 = x * x, y2 = y * y, z2 = z * z, x3 = x2 * x, y3 = y2 * y, z3 = z2 * z;\n"
        "    const real x4 = x2 * x2, y4 = y2 * y2, z4 = z2 * z2;\n"
        "    (void)x3; (void)y3; (void)z3; (void)x4; (void)y4; (void)z4;")


def emit():
    out = []
    out.append("// Generated by gen_sh.py -- real orthonormal spherical harmonics, l = 1..4.")
    out.append("// Index k = l*l - 1 + (m + l); each Y_k is a homogeneous harmonic polynomial of")
    out.append("// degree l in the components of the unit vector (x, y, z).")
    out.append("#pragma once")
    out.append("")
    out.append("template <typename real>")
    out.append("__device__ __forceinline__ void sh_eval(real x, real y, real z, real* Y)")
    out.append("{")
    out.append(MONO)
    for i, k in enumerate(KEYS):
        out.append(f"    Y[{i}] = {c(Y[k])};")
    out.append("}")
    return "\n".join(out) + "\n"


# The sphere-reduced form: with z^2 = 1 - x^2 - y^2 (exact on the unit sphere) every
# Y_k is A_k(x, y) + z B_k(x, y), deg A_k <= 4, deg B_k <= 3.  Coefficient layout of
# a 25-entry vector: block A (x^a y^b, a + b <= 4) at red_a(a) + b, then block B
# (z x^a y^b, a + b <= 3) at red_b(a) + b.
RED_A = [(a, b) for a in range(5) for b in range(5 - a)]
RED_B = [(a, b) for a in range(4) for b in range(4 - a)]


def reduced(v):
    """(A coefficients, B coefficients) of the reduced form of polynomial v."""
    rem = sp.expand(sp.rem(sp.expand(v), z * z - (1 - x * x - y * y), z))
    p = sp.Poly(rem, x, y, z)
    assert p.degree(z) <= 1
    ca = [p.coeff_monomial(x ** a * y ** b) for a, b in RED_A]
    cb = [p.coeff_monomial(x ** a * y ** b * z) for a, b in RED_B]
    return ca, cb


def check_reduced():
    """On random points of the sphere the reduced form equals Y_k, and its gradient
    differs from grad Y_k only along the normal (equal surface gradients)."""
    rng = np.random.default_rng(7)
    u = rng.standard_normal((3, 200))
    u /= np.linalg.norm(u, axis=0)
    for k in KEYS:
        ca, cb = reduced(Y[k])
        red = sum(c * x ** a * y ** b for c, (a, b) in zip(ca, RED_A)) + \
            z * sum(c * x ** a * y ** b for c, (a, b) in zip(cb, RED_B))
        f = sp.lambdify((x, y, z), Y[k] - red, "numpy")
        assert np.abs(f(*u) * np.ones(u.shape[1])).max() < 1e-12
        g = np.array([sp.lambdify((x, y, z), sp.diff(Y[k] - red, w), "numpy")(*u) * np.ones(u.shape[1])
                      for w in (x, y, z)])
        tang = g - (g * u).sum(axis=0) * u
        assert np.abs(tang).max() < 1e-12


def emit_reduced():
    out = []
    out.append("")
    out.append("// Sphere-reduced form: with z^2 = 1 - x^2 - y^2 each Y_k equals A_k(x, y) + z B_k(x, y)")
    out.append("// on the unit sphere, deg A_k <= 4, deg B_k <= 3 (the two forms have equal values and")
    out.append("// equal surface gradients there).  A 25-entry coefficient vector holds block A")
    out.append("// (x^a y^b, a + b <= 4) at sh_red_a(a) + b and block B (z x^a y^b, a + b <= 3) at")
    out.append("// sh_red_b(a) + b.")
    out.append(f"constexpr int kShRed = {len(RED_A) + len(RED_B)};")
    out.append("__host__ __device__ constexpr int sh_red_a(int a) { return a * 5 - a * (a - 1) / 2; }")
    out.append(f"__host__ __device__ constexpr int sh_red_b(int a) {{ return {len(RED_A)} + a * 4 - a * (a - 1) / 2; }}")
    out.append("")
    out.append("// psi = sum_k phi[k] (reduced form of Y_k): the reduced coefficients of sum_k phi[k] Y_k")
    out.append("template <typename real>")
    out.append("__device__ __forceinline__ void sh_reduce(const real* phi, real* psi)")
    out.append("{")
    cols = [reduced(Y[k]) for k in KEYS]
    for j, (a, b) in enumerate(RED_A + RED_B):
        blk = 0 if j < len(RED_A) else 1
        jj = j if blk == 0 else j - len(RED_A)
        terms = []
        for i, (ca, cb) in enumerate(cols):
            cf = (ca if blk == 0 else cb)[jj]
            if cf != 0:
                terms.append(f"real({sp.N(cf, 17)}) * phi[{i}]")
        out.append(f"    psi[{j}] = {' + '.join(terms) if terms else 'real(0)'};")
    out.append("}")
    return "\n".join(out) + "\n"


if __name__ == "__main__":
    check()
    check_reduced()
    sys.stdout.write(emit())
    sys.stdout.write(emit_reduced())
