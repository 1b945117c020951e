"""HNEMD steps through the C ABI: FP64 trajectory and heat-current rows equal the
oracle's (driving force, with and without the thermostat), the interval averages
of the rows, graph replay equal to eager launches, and a zero field equal to the
plain MD step."""
import numpy as np
import pytest

import oracle
from paper_2603_01234_gb300 import binding, inputs
from tests.gpu_common import water_model

pytestmark = pytest.mark.gpu


def state(n=256, seed=41, T=300.0):
    s = inputs.water_box(n, seed=seed)
    s.masses = np.array([18.0])
    v = inputs.maxwell_boltzmann(s, T, seed=seed + 1)
    return s, v


@pytest.mark.parametrize("thermostat", [False, True])
def test_fp64_hnemd_matches_oracle(nep_lib, thermostat):
    model = water_model()
    s, v = state()
    steps, dt, every = 20, 2.0, 5
    fe = np.array([0.0, 0.01, 0.03])
    T, tau = 320.0, 30.0
    noise = binding.bussi_noise(steps, s.n, seed=43) if thermostat else None
    r0 = oracle.compute(model, s)
    f0 = oracle.hnemd_force(fe, r0.virial, r0.force)
    p_ref, v_ref, f_ref, th_ref, heat_ref = oracle.md(model, s, s.pos, v, f0, steps, dt, temperature=T, tau=tau,
                                                      noise=noise, fe=fe)
    m = binding.Model(model, "fp64")
    pos, vel, force = s.pos.copy(), v.copy(), np.zeros_like(s.pos)
    thermo = np.zeros((steps // every, 12))
    heat = np.zeros((steps // every, 6))
    binding.nep_md_step_hnemd(m.h, s.types, s.masses, s.box, s.pbc, pos, vel, force, 0, steps, dt, fe, T, tau,
                              noise, every, thermo, heat)
    np.testing.assert_allclose(pos, p_ref, atol=1e-9)
    np.testing.assert_allclose(vel, v_ref, atol=1e-11)
    np.testing.assert_allclose(force, f_ref, atol=1e-9)
    np.testing.assert_allclose(thermo[:, 2], th_ref[every - 1::every, 1], rtol=1e-10, atol=1e-12)
    want = heat_ref.reshape(steps // every, every, 6).mean(axis=1)
    scale = np.abs(heat_ref).max(axis=0)
    assert np.all(np.abs(heat - want) <= 1e-9 * scale + 1e-14), np.abs(heat - want).max(axis=0)
    m.close()


def test_fp32_first_step_heat_current(nep_lib):
    model = water_model()
    s, v = state(n=1000, seed=44)
    fe = np.array([0.02, 0.0, 0.0])
    r0 = oracle.compute(model, s)
    f0 = oracle.hnemd_force(fe, r0.virial, r0.force)
    _, v_ref, f_ref, _, heat_ref = oracle.md(model, s, s.pos, v, f0, 1, 1.0, fe=fe)
    m = binding.Model(model, "fp32")
    pos, vel, force = s.pos.copy(), v.copy(), np.zeros_like(s.pos)
    heat, thermo = np.zeros((1, 6)), np.zeros((1, 12))
    binding.nep_md_step_hnemd(m.h, s.types, s.masses, s.box, s.pbc, pos, vel, force, 0, 1, 1.0, fe,
                              sample_every=1, thermo=thermo, heat=heat)
    # J_pot = sum_i W_i v_i: each term carries the FP32 virial tolerance 1e-4 W_rms
    wscale = np.sqrt((r0.virial ** 2).mean()) * np.abs(v_ref).sum(axis=1)
    assert np.all(np.abs(heat[0, :3] - heat_ref[0, :3]) <= 1e-4 * wscale * 3), (heat[0], heat_ref[0])
    uscale = (1 + np.abs(r0.site_energy)).mean() * np.abs(v_ref).sum(axis=1)
    assert np.all(np.abs(heat[0, 3:] - heat_ref[0, 3:]) <= 1e-5 * uscale), (heat[0], heat_ref[0])
    fscale = np.sqrt((f_ref ** 2).mean())
    assert np.abs(force - f_ref).max() <= 1e-4 * fscale + 1e-6
    m.close()


def test_hnemd_graph_replay_equals_eager(nep_lib):
    model = water_model()
    s, v = state(n=500, seed=45)
    fe = np.array([0.0, 0.0, 0.02])
    noise = binding.bussi_noise(20, s.n, seed=46)
    runs = []
    for mode in ("graph", "eager"):
        m = binding.Model(model, "fp32")
        if mode == "eager":
            binding.nep_set_timing(m.h, 1)
        pos, vel, force = s.pos.copy(), v.copy(), np.zeros_like(s.pos)
        th, heat = np.zeros((4, 12)), np.zeros((4, 6))
        binding.nep_md_step_hnemd(m.h, s.types, s.masses, s.box, s.pbc, pos, vel, force, 0, 20, 4.0, fe, 300.0,
                                  50.0, noise, 5, th, heat)
        runs.append((pos, vel, force, th, heat))
        m.close()
    for a, b in zip(runs[0], runs[1]):
        np.testing.assert_array_equal(a, b)


def test_zero_field_equals_plain_md(nep_lib):
    model = water_model()
    s, v = state(n=400, seed=47)
    out = []
    for drive in (False, True):
        m = binding.Model(model, "fp32")
        pos, vel, force = s.pos.copy(), v.copy(), np.zeros_like(s.pos)
        th = np.zeros((3, 12))
        if drive:
            heat = np.zeros((3, 6))
            binding.nep_md_step_hnemd(m.h, s.types, s.masses, s.box, s.pbc, pos, vel, force, 0, 15, 4.0,
                                      np.zeros(3), sample_every=5, thermo=th, heat=heat)
            assert np.all(np.isfinite(heat)) and np.abs(heat).max() > 0
        else:
            binding.nep_md_step(m.h, s.types, s.masses, s.box, s.pbc, pos, vel, force, 0, 15, 4.0, 5, th)
        out.append((pos, vel, th))
        m.close()
    for a, b in zip(out[0], out[1]):
        np.testing.assert_array_equal(a, b)


def test_hnemd_argument_errors(nep_lib):
    model = water_model()
    s, v = state(n=100, seed=48)
    m = binding.Model(model, "fp32")
    pos, vel, force = s.pos.copy(), v.copy(), np.zeros_like(s.pos)
    with pytest.raises(binding.NepError) as e:
        binding.nep_md_step_hnemd(m.h, s.types, s.masses, s.box, s.pbc, pos, vel, force, 0, 4, 1.0,
                                  np.array([0.0, np.nan, 0.0]))
    assert e.value.code == binding.NEP_ERR_ARG
    with pytest.raises(binding.NepError) as e:  # heat rows need a sampling interval
        binding.nep_md_step_hnemd(m.h, s.types, s.masses, s.box, s.pbc, pos, vel, force, 0, 4, 1.0,
                                  np.zeros(3), heat=np.zeros((1, 6)))
    assert e.value.code == binding.NEP_ERR_ARG
    m.close()
