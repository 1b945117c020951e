"""nep_compute_static, the evaluation that allocates no device memory, through the
C ABI.

Some callers cannot let a library allocate device memory: engines that budget all
GPU memory at start-up, loops that cannot absorb the device-wide synchronisation
of cudaFree, processes where an allocation failing mid-run is unacceptable.  For
them nep_compute_static takes its scratch from one fixed array in the library
image.  It runs the same kernels in the same order as nep_compute, so its results
must be bitwise equal to nep_compute's; two calls in a row with different sizes
check that nothing the first call leaves in the shared array reaches the second.
One small system is also compared with the FP64 oracle.  This file sorts last so
that a run that stops at the first failure has run every other test first.
"""
import numpy as np
import pytest

import oracle
from paper_2603_01234_gb300 import binding, inputs
from tests.gpu_common import assert_parity, water_model

pytestmark = pytest.mark.gpu

KEYS = ("energy", "virial_total", "site_energy", "force", "virial")


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


def _assert_bitwise(got, ref):
    for k in KEYS:
        assert np.array_equal(got[k], ref[k]), (k, np.abs(got[k] - ref[k]).max())


def test_static_scratch_bitwise_equal_to_nep_compute_twice():
    import torch
    binding.load(build_if_missing=True)
    dev = torch.device("cuda:0")
    m = binding.Model(water_model(), "fp32")
    first = inputs.water_box(3000, seed=21)
    second = inputs.water_box(700, seed=22)
    for system in (first, second):
        ref = _run(torch, binding.nep_compute, m, system, dev)
        got = _run(torch, binding.nep_compute_static, m, system, dev)
        _assert_bitwise(got, ref)
    m.close()


def test_static_scratch_matches_oracle():
    import torch
    binding.load(build_if_missing=True)
    dev = torch.device("cuda:0")
    model = water_model(seed=9)
    system = inputs.water_box(1000, seed=10)
    for precision in ("fp32", "fp64"):
        m = binding.Model(model, precision)
        got = _run(torch, binding.nep_compute_static, m, system, dev)
        m.close()
        got["energy"] = float(got["energy"][0])
        assert_parity(got, oracle.compute(model, system), precision)


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
    _assert_bitwise(got, ref)
    m.close()
