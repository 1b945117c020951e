"""The FP32 screening of the FP64 neighbour search decides every distance test as the
FP64 test does.  The kernel's FP32 arithmetic is emulated here in numpy (each FP32
operation rounded once, multiply-adds fused as the compiler fuses them), with the
screening bounds formed as the kernel forms them, on pairs drawn close to the cutoff
anywhere in the coordinate range the bound covers (cell-relative coordinates within
two cell lengths of the cell's origin)."""
import numpy as np

F32 = np.float32


def f32(x):
    return np.asarray(x, dtype=np.float64).astype(F32)


def round_down(v):
    r = f32(v)
    return np.where(r.astype(np.float64) > v, np.nextafter(r, F32(-np.inf)), r)


def round_up(v):
    r = f32(v)
    return np.where(r.astype(np.float64) < v, np.nextafter(r, F32(np.inf)), r)


def bounds(c2, lmax):
    """The kernel's screening bounds (lo, hi) for a squared cutoff c2."""
    d = np.sqrt(3.0) * lmax * 2.0 ** -19
    eps = 4.0 * (2.0 * np.sqrt(c2) * d + d * d + 3.0 * 2.0 ** -24 * c2)
    return round_down(c2 - eps), round_up(c2 + eps)


def screened_and_exact(rng, n, rc, lens, spread):
    lens = np.asarray(lens, dtype=np.float64)
    lmax = lens.max()
    c2 = rc * rc
    lo, hi = bounds(c2, lmax)
    off = rng.integers(-2, 3, size=(3, n)).astype(np.float64)  # cell offsets dx, dy, dz
    ri = rng.uniform(-2.0, 2.0, size=(3, n)) * lens[:, None] * 0.995
    # j placed at a distance within `spread` (relative) of the cutoff from i's image point
    u = rng.standard_normal((3, n))
    u /= np.linalg.norm(u, axis=0)
    r = rc * (1.0 + rng.uniform(-spread, spread, size=n))
    b = ri - off * lens[:, None]
    rj = b + r * u
    keep = np.all(np.abs(rj) <= 1.99 * lens[:, None], axis=0)  # the range the bound covers
    ri, rj, off, b = ri[:, keep], rj[:, keep], off[:, keep], b[:, keep]
    # FP64 test, as the kernel's FP64 path computes it
    dd = rj - b
    r2 = (dd * dd).sum(axis=0)
    exact = r2 < c2
    # FP32 screen: bxf = fma(-dx, len_f, ri_f), fx = rj_f - bxf, r2f by fused multiply-adds
    lf = f32(lens)[:, None].astype(np.float64)
    bf = f32(f32(ri).astype(np.float64) - off * lf).astype(np.float64)
    fx = f32(f32(rj).astype(np.float64) - bf).astype(np.float64)
    t = f32(fx[0] * fx[0]).astype(np.float64)
    t = f32(fx[1] * fx[1] + t).astype(np.float64)
    r2f = f32(fx[2] * fx[2] + t)
    sure_in = r2f < lo
    maybe_in = r2f < hi
    band = sure_in != maybe_in
    decided = np.where(band, exact, sure_in)
    return decided, exact, band


def test_screen_decides_as_fp64_near_the_cutoff():
    rng = np.random.default_rng(11)
    for rc, lens in ((8.0, (8.006, 8.006, 8.006)), (15.0, (20.0, 18.19, 15.0)), (5.0, (9.9, 5.1, 7.3)),
                     (7.0, (7.0, 13.9, 13.9))):
        # within 1e-3 of the cutoff: both sides of the band and its edges
        decided, exact, band = screened_and_exact(rng, 400_000, rc, lens, 1e-3)
        assert decided.size > 100_000
        assert np.array_equal(decided, exact)
        assert 0.0 < band.mean() < 0.25  # most pairs even this close are decided in FP32
        # a wider draw: the band is left to the FP64 test only for a small fraction
        decided, exact, band = screened_and_exact(rng, 400_000, rc, lens, 0.2)
        assert np.array_equal(decided, exact)
        assert band.mean() < 0.01


def test_screen_bounds_enclose_the_cutoff():
    for rc in (5.0, 8.0, 15.0):
        lo, hi = bounds(rc * rc, 2.0 * rc)
        assert float(lo) < rc * rc < float(hi)
        assert (float(hi) - float(lo)) / (rc * rc) < 2e-4
