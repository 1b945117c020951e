"""Shared helpers of the GPU parity tests: test systems and tolerance checks.

Tolerances (stated here, derived in the design notes):
  FP64 form   every quantity within 1e-10 of the oracle, relative to its scale
  FP32 form   site energy |dU_i| <= 1e-5 (1 + |U_i|)
              total energy |dE| <= 1e-6 sum_i |U_i| (and E equals the FP64 sum of the
              returned U_i to 1e-12: the reduction adds no error of its own)
              forces  max |dF| <= 1e-4 F_rms + 1e-6 eV/A
              virials max |dW_i| <= 1e-4 W_rms + 1e-7 eV;  |dW_tot| <= 1e-5 sum_i |W_i|
"""
import numpy as np

from paper_2603_01234_gb300 import inputs

TOL = {
    "fp64": dict(U=1e-10, E=1e-10, F=1e-10, F_abs=1e-12, W=1e-10, W_abs=1e-12, Wt=1e-10),
    "fp32": dict(U=1e-5, E=1e-6, F=1e-4, F_abs=1e-6, W=1e-4, W_abs=1e-7, Wt=1e-5),
}


def rms(x):
    return float(np.sqrt(np.mean(np.square(x)))) if x.size else 0.0


def assert_parity(got, ref, precision, beads=None):
    """got: dict from binding.Model.compute; ref: oracle.OracleResult."""
    t = TOL[precision]
    sel = slice(None) if beads is None else beads
    U, Ur = got["site_energy"][sel], ref.site_energy[sel]
    if precision == "fp64":
        assert np.abs(U - Ur).max() <= t["U"] * (1 + np.abs(Ur).max()), np.abs(U - Ur).max()
    else:
        assert np.all(np.abs(U - Ur) <= t["U"] * (1 + np.abs(Ur))), np.abs(U - Ur).max()
    F, Fr = got["force"][:, sel], ref.force[:, sel]
    fs = rms(ref.force[:, sel]) if precision == "fp32" else np.abs(Fr).max()
    assert np.abs(F - Fr).max() <= t["F"] * fs + t["F_abs"], (np.abs(F - Fr).max(), fs)
    W, Wr = got["virial"][:, sel], ref.virial[:, sel]
    ws = rms(Wr) if precision == "fp32" else np.abs(Wr).max()
    assert np.abs(W - Wr).max() <= t["W"] * ws + t["W_abs"], (np.abs(W - Wr).max(), ws)
    if beads is None:
        # the FP64 reduction adds no error of its own: E is the sum of the returned U_i
        usum = got["site_energy"].sum()
        assert abs(got["energy"] - usum) <= 1e-12 * np.abs(got["site_energy"]).sum() + 1e-14
        escale = np.abs(ref.site_energy).sum()
        assert abs(got["energy"] - ref.energy) <= t["E"] * escale + 1e-12, (got["energy"], ref.energy, escale)
        wscale = np.abs(ref.virial).sum()
        assert np.abs(got["virial_total"] - ref.virial_total).max() <= t["Wt"] * wscale + 1e-12


# ---- test systems (small enough for the oracle in seconds) ---------------------
def water_model(seed=1, hidden=30):
    return inputs.random_model(n_types=1, hidden=hidden, rc_radial=8.0, rc_angular=5.0, seed=seed)


def monolayer_model(seed=2):
    return inputs.random_model(n_types=4, hidden=50, rc_radial=15.0, rc_angular=11.0, seed=seed)


def aacg_model(seed=3):
    """Two particle types with per-pair cutoffs: 6/5 A (atom-atom), 8/7 A
    (bead-bead) and their means 7/6 A for mixed pairs (Sec. III.C)."""
    return inputs.random_model(n_types=2, hidden=30, rc_radial=inputs.pair_table(2, [6.0, 8.0]),
                               rc_angular=inputs.pair_table(2, [5.0, 7.0]), seed=seed)


def nanowire_model(seed=4):
    return inputs.random_model(n_types=3, hidden=40, rc_radial=7.0, rc_angular=5.0, seed=seed)


def small_systems():
    """(name, model, system) cases spanning several tiles and ragged tails."""
    yield "water512", water_model(), inputs.water_small()
    yield "water64_images", water_model(seed=5), inputs.water_box(64, seed=6)
    yield "water37_tiny_box", water_model(seed=7), inputs.water_box(37, seed=8)
    # 1, 2 and 3 cells per periodic axis: every stencil row wraps and repeats cells as images
    yield "box6x9x13_images", water_model(seed=16), inputs.random_periodic(8, [6.0, 9.0, 13.0], seed=17,
                                                                             min_dist=1.5)
    yield "water1000", water_model(seed=9), inputs.water_box(1000, seed=10)
    yield "monolayer4types", monolayer_model(), inputs.monolayer(6, 5, seed=11)
    s = inputs.random_periodic(300, [16.0, 17.0, 18.0], seed=12, min_dist=1.4, n_types=2)
    yield "aacg300", aacg_model(), s
    w = inputs.nanowire(n_total=3000, n_cells_x=12, seed=13, margin=5.0)
    yield "nanowire3000", nanowire_model(), w
    # six types with per-pair cutoffs (means of per-type values) and a ragged tail
    m6 = inputs.random_model(n_types=6, hidden=24, rc_radial=inputs.pair_table(6, [5.0, 5.5, 6.0, 6.5, 7.0, 7.5]),
                             rc_angular=inputs.pair_table(6, [4.0, 4.2, 4.4, 4.6, 4.8, 5.0]), seed=18)
    yield "mix6types", m6, inputs.random_periodic(333, [17.0, 18.0, 19.0], seed=19, min_dist=1.5, n_types=6)
    # the second compiled shape: n_R = n_A = 5, K_R = K_A = 9 (n_A not a multiple of 4)
    m = inputs.random_model(n_types=2, n_desc_radial=5, n_desc_angular=5, n_basis_radial=9, n_basis_angular=9,
                            hidden=20, rc_radial=6.0, rc_angular=4.5, seed=14)
    yield "shape5599_2types", m, inputs.random_periodic(400, [18.0, 18.0, 18.0], seed=15, min_dist=1.6, n_types=2)
