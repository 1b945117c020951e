"""CUDA path vs the FP64 oracle on the same seeded inputs, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_2603_01234_gb300 import binding, inputs
from tests.gpu_common import assert_parity, small_systems, water_model

pytestmark = pytest.mark.gpu

CASES = list(small_systems())
IDS = [c[0] for c in CASES]


def pair_sets(nb, kind, system, model, band):
    """Oracle pairs of one kind, split into certain and near-cutoff (|r - rc| < band)."""
    col = 5 + kind
    rows = nb[nb[:, col] == 1]
    w = oracle.wrap(system)
    d = (w[:, rows[:, 1]] + rows[:, 2:5].T * system.box[:, None]) - w[:, rows[:, 0]]
    r = np.sqrt((d * d).sum(axis=0))
    rc_tab = model.rc_radial if kind == 0 else model.rc_angular
    rc = rc_tab[system.types[rows[:, 0]], system.types[rows[:, 1]]]
    near = np.abs(r - rc) < band
    return set(map(tuple, rows[~near][:, :5])), set(map(tuple, rows[near][:, :5]))


@pytest.mark.parametrize("name,model,system", CASES, ids=IDS)
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_neighbor_sets_match_brute_force(nep_lib, name, model, system, precision):
    m = binding.Model(model, precision)
    nb = oracle.neighbors(model, system, use_cells=False)
    band = 1e-4 if precision == "fp32" else 1e-9
    for kind in (0, 1):
        cnt, j, sh = m.neighbors(system, kind=kind, capacity=512)
        got = set()
        for i in range(system.n):
            assert cnt[i] <= 512
            for s in range(cnt[i]):
                got.add((i, int(j[i, s]), *map(int, sh[i, s])))
        assert len(got) == int(cnt.sum())  # no duplicate (j, image) entries
        certain, near = pair_sets(nb, kind, system, model, band)
        assert certain <= got
        assert got - certain <= near
    m.close()


@pytest.mark.parametrize("name,model,system", CASES, ids=IDS)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_energy_force_virial_parity(nep_lib, name, model, system, precision):
    ref = oracle.compute(model, system)
    m = binding.Model(model, precision)
    got = m.compute(system)
    assert_parity(got, ref, precision)
    m.close()


def test_translation_and_wrapping(nep_lib):
    """Positions outside the box on periodic axes give the same result."""
    model, system = water_model(), inputs.water_small()
    m = binding.Model(model, "fp64")
    a = m.compute(system)
    s2 = inputs.System(pos=system.pos + np.array([[24.8 * 3], [-24.8 * 2], [24.8 * 7]]), types=system.types,
                       box=system.box, pbc=system.pbc)
    b = m.compute(s2)
    assert b["energy"] == pytest.approx(a["energy"], rel=1e-12)
    np.testing.assert_allclose(b["force"], a["force"], atol=1e-11)


def test_device_mode_equals_host_mode(nep_lib):
    import torch
    model, system = water_model(), inputs.water_box(1000, seed=10)
    m = binding.Model(model, "fp32")
    host = m.compute(system)
    dev = torch.device("cuda:0")
    types = torch.from_numpy(system.types).to(dev)
    pos = torch.from_numpy(system.pos).to(dev)
    out = m.compute_device(types, pos, system.box, system.pbc)
    torch.cuda.synchronize()
    assert float(out["energy"].cpu()[0]) == host["energy"]
    np.testing.assert_array_equal(out["force"].cpu().numpy(), host["force"])
    np.testing.assert_array_equal(out["virial"].cpu().numpy(), host["virial"])
    m.close()


def test_deterministic(nep_lib):
    model, system = water_model(), inputs.water_box(2000, seed=14)
    m = binding.Model(model, "fp32")
    a, b = m.compute(system), m.compute(system)
    assert a["energy"] == b["energy"]
    np.testing.assert_array_equal(a["force"], b["force"])
    np.testing.assert_array_equal(a["virial"], b["virial"])
    m.close()


def test_capacity_regrowth(nep_lib):
    model, system = water_model(), inputs.water_small()
    m = binding.Model(model, "fp64")
    binding.nep_set_capacity(m.h, 8, 8)
    got = m.compute(system)
    r, a = binding.nep_get_capacity(m.h)
    assert r > 8 and a > 8
    assert_parity(got, oracle.compute(model, system), "fp64")
    m.close()


def test_error_paths(nep_lib):
    model, system = water_model(), inputs.water_small()
    m = binding.Model(model, "fp32")
    bad = inputs.System(pos=system.pos, types=system.types.copy(), box=system.box, pbc=system.pbc)
    bad.types[3] = 5
    with pytest.raises(binding.NepError) as e:
        m.compute(bad)
    assert e.value.code == binding.NEP_ERR_ARG
    tiny = inputs.System(pos=system.pos[:, :2].copy() * 0.1, types=system.types[:2], box=np.array([3.0, 3.0, 3.0]),
                         pbc=system.pbc)
    with pytest.raises(binding.NepError) as e:
        m.compute(tiny)
    assert e.value.code == binding.NEP_ERR_BOX_TOO_SMALL
    nanpos = system.pos.copy()
    nanpos[0, 0] = np.nan
    with pytest.raises(binding.NepError) as e:
        m.compute(inputs.System(pos=nanpos, types=system.types, box=system.box, pbc=system.pbc))
    assert e.value.code == binding.NEP_ERR_ARG
    # the handle stays usable after errors
    assert_parity(m.compute(system), oracle.compute(model, system), "fp32")
    m.close()


def test_kernel_variants_identical_and_autotune(nep_lib):
    """Register-cap and walk-chunk variants compute the same numbers bit for bit; the
    autotuner picks one."""
    model, system = water_model(), inputs.water_box(3000, seed=17)
    m = binding.Model(model, "fp32")
    ref = None
    for md_ in (2, 3):
        for mf in (3, 4, 5):
            for ch in (4, 8):
                binding.nep_set_tuning(m.h, 0, md_, mf, ch)
                got = m.compute(system)
                if ref is None:
                    ref = got
                else:
                    np.testing.assert_array_equal(got["force"], ref["force"])
                    np.testing.assert_array_equal(got["virial"], ref["virial"])
                    assert got["energy"] == ref["energy"]
    for bad in ((4, 3, 4), (3, 6, 4), (3, 2, 4), (1, 3, 4), (3, 3, 6), (3, 3, 2)):
        with pytest.raises(binding.NepError):
            binding.nep_set_tuning(m.h, 0, *bad)
    md_, mf, ch = binding.nep_autotune(m.h, system.types, system.pos, system.box, system.pbc)
    assert md_ in (2, 3) and mf in (3, 4, 5) and ch in (4, 8)
    assert binding.nep_get_tuning(m.h) == (md_, mf, ch)
    m.close()
