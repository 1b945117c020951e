"""Velocity-Verlet MD through the C ABI: FP64 trajectory parity with the oracle,
graph replay equal to eager launches, device mode equal to host mode, and NVE
energy conservation of the FP32 form."""
import numpy as np
import pytest

import oracle
from paper_2603_01234_gb300 import binding, inputs
from tests.gpu_common import water_model

pytestmark = pytest.mark.gpu


def state(n=256, seed=3, T=300.0):
    s = inputs.water_box(n, seed=seed)
    s.masses = np.array([18.0])
    v = inputs.maxwell_boltzmann(s, T, seed=seed + 1)
    return s, v


def test_fp64_trajectory_matches_oracle(nep_lib):
    model = water_model()
    s, v = state()
    steps, dt = 20, 2.0
    f0 = oracle.compute(model, s).force
    p_ref, v_ref, f_ref, th_ref = oracle.md(model, s, s.pos, v, f0, steps, dt)
    m = binding.Model(model, "fp64")
    pos, vel, force = s.pos.copy(), v.copy(), np.zeros_like(s.pos)
    thermo = np.zeros((steps, 12))
    binding.nep_md_step(m.h, s.types, s.masses, s.box, s.pbc, pos, vel, force, 0, steps, dt, 1, thermo)
    np.testing.assert_allclose(pos, p_ref, atol=1e-9)
    np.testing.assert_allclose(vel, v_ref, atol=1e-11)
    np.testing.assert_allclose(force, f_ref, atol=1e-9)
    np.testing.assert_allclose(thermo[:, 1], th_ref[:, 0], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(thermo[:, 2], th_ref[:, 1], rtol=1e-10, atol=1e-12)
    np.testing.assert_array_equal(thermo[:, 0], np.arange(1, steps + 1))
    m.close()


def test_fp64_trajectory_with_deferred_kicks_matches_oracle(nep_lib):
    """A thermo row every 5 steps lets the steps in between defer their closing kick
    into the next step's opening kernel (and the sampled and last steps apply it in
    the output pass); the trajectory still equals the oracle's plain velocity-Verlet
    one."""
    model = water_model()
    s, v = state(n=300, seed=13)
    steps, dt = 20, 2.0
    f0 = oracle.compute(model, s).force
    p_ref, v_ref, f_ref, th_ref = oracle.md(model, s, s.pos, v, f0, steps, dt)
    m = binding.Model(model, "fp64")
    pos, vel, force = s.pos.copy(), v.copy(), np.zeros_like(s.pos)
    thermo = np.zeros((steps // 5, 12))
    binding.nep_md_step(m.h, s.types, s.masses, s.box, s.pbc, pos, vel, force, 0, steps, dt, 5, thermo)
    np.testing.assert_allclose(pos, p_ref, atol=1e-9)
    np.testing.assert_allclose(vel, v_ref, atol=1e-11)
    np.testing.assert_allclose(force, f_ref, atol=1e-9)
    np.testing.assert_allclose(thermo[:, 1], th_ref[4::5, 0], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(thermo[:, 2], th_ref[4::5, 1], rtol=1e-10, atol=1e-12)
    np.testing.assert_array_equal(thermo[:, 0], [5, 10, 15, 20])
    m.close()


def test_graph_replay_equals_eager(nep_lib):
    model = water_model()
    s, v = state(n=500, seed=5)
    runs = []
    for mode in ("graph", "eager"):
        m = binding.Model(model, "fp32")
        pos, vel, force = s.pos.copy(), v.copy(), np.zeros_like(s.pos)
        if mode == "graph":  # one call: chunks of 5 steps captured and replayed
            th = np.zeros((4, 12))
            binding.nep_md_step(m.h, s.types, s.masses, s.box, s.pbc, pos, vel, force, 0, 20, 5.0, 5, th)
        else:  # stage timing forces eager launches
            binding.nep_set_timing(m.h, 1)
            th = np.zeros((4, 12))
            binding.nep_md_step(m.h, s.types, s.masses, s.box, s.pbc, pos, vel, force, 0, 20, 5.0, 5, th)
            _, steps = binding.nep_get_timing(m.h)
            assert steps == 20
        runs.append((pos, vel, force, th))
        m.close()
    for a, b in zip(runs[0], runs[1]):
        np.testing.assert_array_equal(a, b)


def test_device_async_equals_host(nep_lib):
    import torch
    model = water_model()
    s, v = state(n=700, seed=7)
    m = binding.Model(model, "fp32")
    pos, vel, force = s.pos.copy(), v.copy(), np.zeros_like(s.pos)
    binding.nep_md_step(m.h, s.types, s.masses, s.box, s.pbc, pos, vel, force, 0, 12, 5.0)
    m.close()
    m = binding.Model(model, "fp32")
    dev = torch.device("cuda:0")
    t = torch.from_numpy(s.types).to(dev)
    P, V = torch.from_numpy(s.pos.copy()).to(dev), torch.from_numpy(v.copy()).to(dev)
    Fd = torch.zeros_like(P)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        binding.nep_md_step(m.h, t, s.masses, s.box, s.pbc, P, V, Fd, 0, 5, 5.0, stream=st.cuda_stream)
        binding.nep_md_step(m.h, t, s.masses, s.box, s.pbc, P, V, Fd, 1, 7, 5.0, stream=st.cuda_stream)
    binding.nep_sync(m.h)
    st.synchronize()
    np.testing.assert_array_equal(P.cpu().numpy(), pos)
    np.testing.assert_array_equal(V.cpu().numpy(), vel)
    np.testing.assert_array_equal(Fd.cpu().numpy(), force)
    m.close()


def test_fp32_nve_energy_conservation(nep_lib):
    model = water_model()
    s, v = state(n=512, seed=9)
    m = binding.Model(model, "fp32")
    pos, vel, force = s.pos.copy(), v.copy(), np.zeros_like(s.pos)
    th = np.zeros((100, 12))
    binding.nep_md_step(m.h, s.types, s.masses, s.box, s.pbc, pos, vel, force, 0, 1000, 1.0, 10, th)
    etot = th[:, 1] + th[:, 2]
    ke = th[:, 2].mean()
    # fluctuation of the total energy small against the kinetic energy
    assert etot.max() - etot.min() < 2e-3 * ke, (etot.max() - etot.min(), ke)
    m.close()


def test_box_rescale_positions(nep_lib):
    model = water_model()
    s, v = state(n=300, seed=11)
    m = binding.Model(model, "fp32")
    pos = s.pos.copy()
    binding.nep_scale_positions(m.h, pos, [1.001, 1.0, 1.0])
    np.testing.assert_allclose(pos[0], s.pos[0] * 1.001)
    m.close()


def test_fp64_nvt_trajectory_matches_oracle(nep_lib):
    model = water_model()
    s, v = state(n=200, seed=13)
    steps, dt, T, tau = 20, 2.0, 350.0, 20.0
    noise = binding.bussi_noise(steps, s.n, seed=14)
    f0 = oracle.compute(model, s).force
    p_ref, v_ref, f_ref, th_ref = oracle.md(model, s, s.pos, v, f0, steps, dt, temperature=T, tau=tau, noise=noise)
    m = binding.Model(model, "fp64")
    pos, vel, force = s.pos.copy(), v.copy(), np.zeros_like(s.pos)
    thermo = np.zeros((steps, 12))
    binding.nep_md_step_nvt(m.h, s.types, s.masses, s.box, s.pbc, pos, vel, force, 0, steps, dt, T, tau, noise, 1,
                            thermo)
    np.testing.assert_allclose(pos, p_ref, atol=1e-9)
    np.testing.assert_allclose(vel, v_ref, atol=1e-11)
    np.testing.assert_allclose(thermo[:, 2], th_ref[:, 1], rtol=1e-10, atol=1e-12)
    m.close()


def test_fp32_nvt_holds_temperature(nep_lib):
    model = water_model()
    s, v = state(n=1000, seed=15, T=100.0)
    steps, dt, T, tau = 2000, 5.0, 300.0, 100.0
    noise = binding.bussi_noise(steps, s.n, seed=16)
    m = binding.Model(model, "fp32")
    pos, vel, force = s.pos.copy(), v.copy(), np.zeros_like(s.pos)
    th = np.zeros((steps // 10, 12))
    binding.nep_md_step_nvt(m.h, s.types, s.masses, s.box, s.pbc, pos, vel, force, 0, steps, dt, T, tau, noise, 10, th)
    temp = 2.0 * th[:, 2] / ((3 * s.n - 3) * inputs.KB_EV)
    assert abs(temp[len(temp) // 2:].mean() - T) < 0.03 * T, temp[-5:]
    m.close()
