"""The generated headers of the CUDA kernels equal what their generators write now:
poly32.cuh (FP32 cutoff polynomials of Eq. 8, with the generator's own error
checks) and sh_poly.cuh (real orthonormal harmonics, checked for harmonicity and
orthonormality by its generator)."""
import os
import subprocess
import sys

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2603_01234_gb300", "csrc")


def _regenerate(script):
    r = subprocess.run([sys.executable, os.path.join(CSRC, script)], capture_output=True, text=True, cwd=CSRC)
    assert r.returncode == 0, r.stderr
    return r.stdout


def test_cutoff_polynomials_regenerate():
    with open(os.path.join(CSRC, "poly32.cuh")) as f:
        assert _regenerate("gen_poly32.py") == f.read()


def test_cutoff_polynomials_match_eq8():
    """The polynomials against f_c = (1 + cos(pi r / r_c)) / 2 and its derivative,
    evaluated here in FP64 from the committed coefficients."""
    import numpy as np
    sys.path.insert(0, CSRC)
    try:
        import gen_poly32 as gen_cutoff
    finally:
        sys.path.pop(0)
    P, Q = gen_cutoff.coefficients()
    x = np.linspace(0.0, 1.0, 10001)
    y = x - 0.5
    z = y * y
    hf = 0.25 - y * np.polynomial.polynomial.polyval(z, P.astype(np.float64))
    q = np.polynomial.polynomial.polyval(z, Q.astype(np.float64))
    assert np.abs(2 * hf - 0.5 * (1 + np.cos(np.pi * x))).max() < 1e-7
    assert np.abs(q - np.pi / 4 * np.sin(np.pi * x)).max() < 2e-7
    assert abs(2 * hf[0] - 1.0) < 1e-7 and abs(hf[-1]) < 1e-7  # f_c(0) = 1, f_c(r_c) = 0


def test_harmonics_regenerate():
    pytest.importorskip("sympy")
    with open(os.path.join(CSRC, "sh_poly.cuh")) as f:
        assert _regenerate("gen_sh.py") == f.read()
