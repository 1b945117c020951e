"""nep_compute_static, the evaluation that allocates no device memory, against
nep_compute on the same inputs, through the C ABI.

Callers that cannot allocate (device memory budgeted at start-up, no device-wide
synchronisation allowed in their loop) use this entry point; its scratch is a
fixed array in the library image.  Two calls in a row, with different sizes, must
each match nep_compute within the FP32 tolerances the other parity tests use, so
that nothing the first call leaves in the shared array leaks into the second.
This file sorts last so that a run that stops at the first failure has run every
other test first.
"""
import numpy as np
import pytest

from paper_2603_01234_gb300 import binding, inputs
from tests.gpu_common import TOL, rms, water_model

pytestmark = pytest.mark.gpu


def _device_outputs(torch, n, dev):
    z = lambda *s: torch.zeros(*s, dtype=torch.float64, device=dev)  # noqa: E731
    return {"energy": z(1), "virial_total": z(9), "site_energy": z(n), "force": z(3, n), "virial": z(9, n)}


def _run(torch, fn, m, system, dev):
    types = torch.from_numpy(system.types).to(dev)
    pos = torch.from_numpy(system.pos).to(dev)
    out = _device_outputs(torch, system.n, dev)
    fn(m.h, types, pos, system.box, system.pbc, out["energy"], out["virial_total"], out["site_energy"],
       out["force"], out["virial"])
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _close(a, b):
    t = TOL["fp32"]
    np.testing.assert_allclose(a["site_energy"], b["site_energy"], rtol=0, atol=t["U"] * (1 + np.abs(b["site_energy"]).max()))
    assert np.abs(a["force"] - b["force"]).max() <= t["F"] * rms(b["force"]) + t["F_abs"]
    assert np.abs(a["virial"] - b["virial"]).max() <= t["W"] * rms(b["virial"]) + t["W_abs"]
    assert abs(a["energy"][0] - b["energy"][0]) <= (t["U"] * (1 + np.abs(b["site_energy"]))).sum()
    assert np.abs(a["virial_total"] - b["virial_total"]).max() <= t["Wt"] * np.abs(b["virial"]).sum() + 1e-12


def test_static_scratch_matches_nep_compute_twice():
    import torch
    binding.load(build_if_missing=True)
    dev = torch.device("cuda:0")
    m = binding.Model(water_model(), "fp32")
    first = inputs.water_box(3000, seed=21)
    second = inputs.water_box(700, seed=22)
    for system in (first, second):
        ref = _run(torch, binding.nep_compute, m, system, dev)
        got = _run(torch, binding.nep_compute_static, m, system, dev)
        _close(got, ref)
    m.close()


def test_static_scratch_rejects_oversize():
    import torch
    binding.load(build_if_missing=True)
    dev = torch.device("cuda:0")
    m = binding.Model(water_model(), "fp32")
    big = inputs.water_box(5000, seed=23)
    with pytest.raises(binding.NepError) as e:
        _run(torch, binding.nep_compute_static, m, big, dev)
    assert e.value.code == binding.NEP_ERR_ARG and "4096" in str(e.value)
    m.close()


def test_static_scratch_with_four_and_five_body_terms():
    import torch
    binding.load(build_if_missing=True)
    dev = torch.device("cuda:0")
    p = inputs.random_model(n_types=2, hidden=30, rc_radial=7.0, rc_angular=5.0, seed=24, l_max_4b=2, l_max_5b=1)
    m = binding.Model(p, "fp32")
    system = inputs.random_periodic(2500, [30.0, 30.0, 30.0], seed=25, min_dist=1.5, n_types=2)
    ref = _run(torch, binding.nep_compute, m, system, dev)
    got = _run(torch, binding.nep_compute_static, m, system, dev)
    _close(got, ref)
    m.close()
