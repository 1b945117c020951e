"""Generate poly32.cuh: FP32 polynomials for the cosine cutoff of Eq. 8 and its
derivative, used by the FP32 kernels in place of the hardware sine/cosine, and for
tanh on [-1, 1] (the activation of Eq. 2).

With x = r / r_c in [0, 1] and y = x - 1/2 in [-1/2, 1/2]:
    f_c / 2  = 1/4 + 1/4 cos(pi x) = 1/4 - y P(y^2),   P(z) ~ sin(pi y) / (4 y)
    f_c' / 2 = -(pi / 4) sin(pi x) / r_c = -Q(y^2) / r_c,   Q(z) ~ (pi / 4) cos(pi y)

The hardware approximations of sin and cos carry an error of about 1e-7 that has
a consistent sign over the arguments a neighbour list produces; summed over the
pairs and beads of a configuration it biases the total energy.  These
polynomials are fitted by least squares at Chebyshev nodes on [-1/2, 1/2], one
coefficient at a time in FP32, so that each later coefficient absorbs the
rounding of the earlier ones; their error then oscillates about zero.  The
script checks, with FP32 Horner evaluation emulated in numpy, that the maximum
error and the mean signed error (weighted by r^2, the density of pairs) stay
below the bounds asserted at the end, and writes the header.

tanh on [0, 1] is x + x^3 R(x^2) with R fitted the same way; each hidden unit's
pre-activation keeps one sign over most particles, so an activation error that
leans one way on part of the range would bias every particle's energy alike.

Run:  python gen_poly32.py > poly32.cuh
"""
import sys

import numpy as np

NCOEF = 5
NTANH = 8


def fit(target, basis_fn, n, nodes):
    coef = []
    for j in range(n):
        resid = target - sum(c * basis_fn(i) for i, c in enumerate(coef))
        A = np.stack([basis_fn(i) for i in range(j, n)], axis=1)
        c, *_ = np.linalg.lstsq(A, resid, rcond=None)
        coef.append(float(np.float32(c[0])))
    return np.array(coef, dtype=np.float32)


def horner32(c, z):
    """FP32 Horner evaluation with one rounding per multiply-add (FMA)."""
    acc = np.full_like(z, c[-1], dtype=np.float32)
    for cc in c[-2::-1]:
        acc = (acc.astype(np.float64) * z + np.float64(cc)).astype(np.float32)
    return acc


def coefficients():
    m = 20000
    y = 0.5 * np.cos(np.pi * (np.arange(m) + 0.5) / m)  # Chebyshev nodes on [-1/2, 1/2]
    z = y * y
    P = fit(np.sin(np.pi * y) / 4, lambda i: y * z ** i, NCOEF, y)
    Q = fit(np.pi / 4 * np.cos(np.pi * y), lambda i: z ** i, NCOEF, y)
    return P, Q


def tanh_coefficients():
    m = 20000
    x = np.cos(np.pi * (np.arange(m) + 0.5) / (2 * m))  # Chebyshev nodes on [0, 1]
    z = x * x
    return fit(np.tanh(x) - x, lambda i: x * z ** (i + 1), NTANH, x)


def check_tanh(R):
    x = np.linspace(0.0, 1.0, 2_000_001).astype(np.float32)
    z = (x.astype(np.float64) * x).astype(np.float32)
    xz = (x.astype(np.float64) * z).astype(np.float32)
    h = (x.astype(np.float64) + xz.astype(np.float64) * horner32(R, z)).astype(np.float32)
    e = h.astype(np.float64) - np.tanh(x.astype(np.float64))
    worst = max(abs(float(e[(x >= a) & (x < a + 0.125)].mean())) for a in np.arange(0.0, 1.0, 0.125))
    assert worst < 1e-9 and np.abs(e).max() < 6e-8, (worst, np.abs(e).max())
    return worst, float(np.abs(e).max())


def check(P, Q):
    x = np.linspace(0.0, 1.0, 4_000_001).astype(np.float32)
    y = (x - np.float32(0.5)).astype(np.float32)  # exact (Sterbenz) for x in [1/4, 1]
    z = (y.astype(np.float64) * y).astype(np.float32)
    hf = (0.25 - y.astype(np.float64) * horner32(P, z)).astype(np.float32)
    q = horner32(Q, z)
    x64 = x.astype(np.float64)
    e_hf = hf - (0.25 + 0.25 * np.cos(np.pi * x64))
    e_q = q - np.pi / 4 * np.sin(np.pi * x64)
    w = x64 ** 2
    stats = {}
    for name, e in (("hf", e_hf), ("q", e_q)):
        stats[name] = (float((e * w).sum() / w.sum()), float(np.abs(e).max()))
    assert abs(stats["hf"][0]) < 1e-9 and stats["hf"][1] < 6e-8, stats
    assert abs(stats["q"][0]) < 5e-9 and stats["q"][1] < 2e-7, stats
    return stats


def main():
    P, Q = coefficients()
    stats = check(P, Q)
    R = tanh_coefficients()
    tstats = check_tanh(R)
    out = sys.stdout
    out.write("// Generated by gen_poly32.py -- do not edit.\n")
    out.write("// FP32 cosine cutoff (Eq. 8): with y = r / r_c - 1/2 and z = y^2,\n")
    out.write("//   f_c / 2 = 1/4 - y P(z),   f_c' / 2 = -Q(z) / r_c.\n")
    out.write("// Least-squares fits at Chebyshev nodes, coefficients fixed one at a time in FP32.\n")
    out.write(f"// Emulated FP32 error: f_c/2 mean signed {stats['hf'][0]:+.1e}, max {stats['hf'][1]:.1e};\n")
    out.write(f"//   Q mean signed {stats['q'][0]:+.1e}, max {stats['q'][1]:.1e} (mean weighted by r^2).\n")
    out.write("// tanh(x) = x + x^3 R(x^2) on [-1, 1], fitted the same way; emulated FP32 error:\n")
    out.write(f"//   max {tstats[1]:.1e}, largest mean signed over eighths of [0, 1] {tstats[0]:.1e}.\n")
    out.write("#pragma once\n\nnamespace nep {\n\n")
    for name, c in (("P", P), ("Q", Q), ("R", R)):
        expr = f"{float(c[-1])!r}f"
        for v in c[-2::-1]:
            expr = f"fmaf({expr}, z, {float(v)!r}f)"
        fn = "tanh_r_poly" if name == "R" else f"cut_{name.lower()}"
        out.write(f"__device__ __forceinline__ float {fn}(float z)\n{{\n    return {expr};\n}}\n\n")
    out.write("}  // namespace nep\n")


if __name__ == "__main__":
    main()
