"""The BF16-weight network form through the C ABI.  W0 (Eq. 2) is rounded to BF16
once; the hidden layer's two products run on tensor cores with every activation
split into two BF16 terms and FP32 accumulation.  So the form must equal the FP32
evaluation of the model with BF16-rounded W0, which the FP64 oracle evaluates
directly, at the FP32 form's tolerances: on every small system (one to four types,
ragged tails, H = 30, 40 and 50, both compiled descriptor shapes).  Against the
unrounded model the differences are those of a 2^-9 relative perturbation of W0,
inside the stated BF16 bounds (1e-2 relative on energies, 2e-2 F_rms on forces).
Bitwise properties of the FP32 form (batch = alone, graph = eager) hold too."""
import numpy as np
import pytest

import oracle
from paper_2603_01234_gb300 import binding, inputs
from tests.gpu_common import assert_parity, monolayer_model, rms, small_systems, water_model

pytestmark = pytest.mark.gpu

CASES = list(small_systems())
IDS = [c[0] for c in CASES]


def bf16_round(x):
    """Round to FP32, then to the nearest BF16 (ties to even)."""
    u = np.asarray(x, dtype=np.float64).astype(np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_model(model):
    m = inputs.ModelParams(**{k: getattr(model, k) for k in model.__dataclass_fields__})
    m.w0 = bf16_round(model.w0)
    return m


def test_bf16_rounding_helper():
    """Values with at most 8 significant bits are kept; ties go to the even neighbour."""
    np.testing.assert_array_equal(bf16_round([1.0, 1.5, -0.75, 3.0]), [1.0, 1.5, -0.75, 3.0])
    one_ulp = 2.0 ** -7  # BF16 spacing at 1
    np.testing.assert_array_equal(bf16_round([1 + one_ulp / 2, 1 + 1.5 * one_ulp]), [1.0, 1 + 2 * one_ulp])


@pytest.mark.parametrize("name,model,system", CASES, ids=IDS)
def test_bf16_equals_fp32_of_rounded_model(nep_lib, name, model, system):
    m = binding.Model(model, "bf16")
    got = m.compute(system)
    m.close()
    assert_parity(got, oracle.compute(bf16_model(model), system), "fp32")
    # and against the unrounded model: the BF16 bounds
    ref = oracle.compute(model, system)
    du = np.abs(got["site_energy"] - ref.site_energy)
    assert np.all(du <= 1e-2 * (1 + np.abs(ref.site_energy))), du.max()
    assert np.abs(got["force"] - ref.force).max() <= 2e-2 * rms(ref.force) + 1e-6


def test_bf16_batch_equals_alone_and_graph_equals_eager(nep_lib):
    models = [water_model(), monolayer_model()]
    handles = [binding.Model(p, "bf16") for p in models]
    systems = [(0, inputs.water_box(300, seed=71)), (1, inputs.monolayer(6, 5, seed=72)),
               (0, inputs.water_box(77, seed=73))]
    req_n, req_box, req_pbc, types, pos = binding.pack_requests([s for _, s in systems])
    n = int(req_n.sum())
    e, wt, F, W = np.zeros(len(systems)), np.zeros((len(systems), 9)), np.zeros(3 * n), np.zeros(9 * n)
    binding.nep_compute_batch([h.h for h in handles], req_n, [k for k, _ in systems], req_box, req_pbc, types, pos,
                              e, wt, None, F, W)
    Fs = binding.unpack_blocks(F, req_n, 3)
    for r, (k, s) in enumerate(systems):
        alone = handles[k].compute(s)
        assert e[r] == alone["energy"]
        np.testing.assert_array_equal(Fs[r], alone["force"])
    for h in handles:
        h.close()
    s = inputs.water_box(500, seed=74)
    s.masses = np.array([18.0])
    v = inputs.maxwell_boltzmann(s, 300.0, seed=75)
    runs = []
    for eager in (False, True):
        m = binding.Model(water_model(), "bf16")
        if eager:
            binding.nep_set_timing(m.h, 1)
        pos, vel, force = s.pos.copy(), v.copy(), np.zeros_like(s.pos)
        th = np.zeros((4, 12))
        binding.nep_md_step(m.h, s.types, s.masses, s.box, s.pbc, pos, vel, force, 0, 20, 5.0, 5, th)
        runs.append((pos, vel, th))
        m.close()
    for x, y in zip(*runs):
        np.testing.assert_array_equal(x, y)
