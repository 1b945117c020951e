"""Full-size systems of the workloads (100,000-bead water, also with the four- and
five-body terms, 200,000-bead four-type monolayer, 1,000,000-particle atom-and-bead
nanowire) through the C ABI in the FP32 form, against the oracle on sampled
particles (the oracle evaluates a sample's neighbourhoods only), plus properties
that hold at any size."""
import numpy as np
import pytest

import oracle
from paper_2603_01234_gb300 import binding, inputs
from tests.gpu_common import TOL, rms

pytestmark = pytest.mark.gpu


def workloads():
    yield ("water100k", inputs.random_model(n_types=1, hidden=30, rc_radial=8.0, rc_angular=5.0, seed=1),
           lambda: inputs.water_box(100_000, seed=1001))
    yield ("monolayer200k", inputs.random_model(n_types=4, hidden=50, rc_radial=15.0, rc_angular=11.0, seed=2),
           lambda: inputs.monolayer(250, 200, seed=1002))
    yield ("nanowire1M", inputs.random_model(n_types=3, hidden=40, rc_radial=7.0, rc_angular=5.0, seed=4),
           lambda: inputs.nanowire(1_000_000, seed=1003))
    # the water workload with the four-body (l = 2) and five-body (l = 1) terms added
    yield ("water100k_4b5b", inputs.random_model(n_types=1, hidden=30, rc_radial=8.0, rc_angular=5.0, seed=5,
                                                 l_max_4b=2, l_max_5b=1),
           lambda: inputs.water_box(100_000, seed=1004))


@pytest.mark.parametrize("name,model,make", list(workloads()), ids=[w[0] for w in workloads()])
def test_fullsize_sampled_parity(nep_lib, name, model, make):
    system = make()
    m = binding.Model(model, "fp32")
    got = m.compute(system)
    m.close()
    rng = np.random.default_rng(7)
    sample = np.sort(rng.choice(system.n, size=48, replace=False))
    ref = oracle.compute(model, system, sample=sample, use_cells=True)
    t = TOL["fp32"]
    U, Ur = got["site_energy"][sample], ref.site_energy[sample]
    assert np.all(np.abs(U - Ur) <= t["U"] * (1 + np.abs(Ur))), np.abs(U - Ur).max()
    # the scales come from the oracle's sample, so that an error that inflates every
    # GPU force or virial cannot widen its own bound
    F, Fr = got["force"][:, sample], ref.force[:, sample]
    fscale = rms(Fr)
    assert np.abs(F - Fr).max() <= t["F"] * fscale + t["F_abs"], (np.abs(F - Fr).max(), fscale)
    W, Wr = got["virial"][:, sample], ref.virial[:, sample]
    wscale = rms(Wr)
    assert np.abs(W - Wr).max() <= t["W"] * wscale + t["W_abs"], (np.abs(W - Wr).max(), wscale)
    # any-size properties: E is the FP64 sum of the U_i; translation invariance
    # (sum F = 0 up to FP32 rounding of each F_i); W_tot symmetric (rotation invariance)
    usum = got["site_energy"].sum()
    assert abs(got["energy"] - usum) <= 1e-12 * np.abs(got["site_energy"]).sum() + 1e-12
    fsum = np.abs(got["force"].sum(axis=1)).max()
    assert fsum <= 1e-6 * np.abs(got["force"]).sum() + 1e-9, fsum
    Wt = got["virial_total"].reshape(3, 3)
    assert np.abs(Wt - Wt.T).max() <= 1e-5 * np.abs(got["virial"]).sum() + 1e-9


@pytest.mark.parametrize("name,model,make", [w for w in workloads() if w[0] in ("water100k", "monolayer200k")],
                         ids=["water100k", "monolayer200k"])
def test_fullsize_total_energy(nep_lib, name, model, make):
    """E over every particle of the full-size system against the oracle's full
    evaluation (a few seconds on the host cores), at the FP32 bound on E."""
    system = make()
    m = binding.Model(model, "fp32")
    got = m.compute(system)
    m.close()
    ref = oracle.compute(model, system, use_cells=True)
    escale = np.abs(ref.site_energy).sum()
    err = abs(got["energy"] - ref.energy)
    assert err <= TOL["fp32"]["E"] * escale, (err, escale, err / escale)
