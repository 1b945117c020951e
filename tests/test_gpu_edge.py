"""Edge cases through the C ABI: a lone particle (no neighbours: q = 0, so Eq. 2
gives U = sum_mu w1 tanh(-b0) - b1 and no force), isolated particles beside
clusters, a pair exactly at the cutoff (excluded: f_c(r_c) = 0), empty inputs
(rejected), and one- and two-particle requests inside a batch."""
import numpy as np
import pytest

import oracle
from paper_2603_01234_gb300 import binding, inputs
from tests.gpu_common import assert_parity, rms

pytestmark = pytest.mark.gpu


def two_type_model():
    return inputs.random_model(n_types=2, hidden=20, rc_radial=6.0, rc_angular=4.0, seed=81)


def lone_energy(model, t):
    """Eq. 2 with every descriptor zero."""
    return float(model.w1[t] @ np.tanh(-model.b0[t]) - model.b1[t])


def system_of(points, types, box=60.0, pbc=(0, 0, 0)):
    return inputs.System(pos=np.ascontiguousarray(np.asarray(points, dtype=np.float64).T),
                         types=np.asarray(types, dtype=np.int32), box=np.array([box] * 3),
                         pbc=np.array(pbc, dtype=np.int32), masses=np.array([12.0, 40.0]))


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_single_particle_closed_form(nep_lib, precision):
    model = two_type_model()
    for t in (0, 1):
        s = system_of([[3.0, 4.0, 5.0]], [t])
        m = binding.Model(model, precision)
        got = m.compute(s)
        m.close()
        want = lone_energy(model, t)
        tol = 1e-12 if precision == "fp64" else 1e-5 * (1 + abs(want))
        assert abs(got["energy"] - want) <= tol, (got["energy"], want)
        assert np.all(got["force"] == 0.0) and np.all(got["virial"] == 0.0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_isolated_particles_beside_clusters(nep_lib, precision):
    model = two_type_model()
    rng = np.random.default_rng(82)
    cluster = inputs.random_cluster(20, seed=83, box_len=7.0, min_dist=1.6, n_types=2)
    pts = list(cluster.pos.T + 10.0) + [[45.0, 45.0, 45.0], [45.0, 5.0, 50.0], [5.0, 50.0, 30.0]]
    types = list(cluster.types) + [0, 1, 1]
    pts += list(cluster.pos.T + np.array([30.0, 10.0, 30.0]))
    types += list(cluster.types)
    order = rng.permutation(len(pts))  # isolated particles anywhere in the caller order
    s = system_of(np.array(pts)[order], np.array(types)[order])
    m = binding.Model(model, precision)
    got = m.compute(s)
    m.close()
    ref = oracle.compute(model, s)
    assert_parity(got, ref, precision)
    lone = [int(np.flatnonzero(order == 20 + q)[0]) for q in range(3)]
    for q, k in enumerate(lone):
        t = [0, 1, 1][q]
        assert abs(got["site_energy"][k] - lone_energy(model, t)) <= 1e-5 * (1 + abs(lone_energy(model, t)))
        assert np.all(got["force"][:, k] == 0.0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_pair_at_the_cutoff(nep_lib, precision):
    """Two particles exactly r_c^R = 8 A apart: f_c and f_c' vanish at r_c, so the
    pair adds (almost) nothing whether or not a rounding of the FP32 pair vector
    puts it just inside the cutoff (one ulp inside, f_c' is about 1e-7)."""
    model = inputs.random_model(n_types=1, hidden=10, rc_radial=8.0, rc_angular=5.0, seed=84)
    s = system_of([[10.0, 20.0, 20.0], [18.0, 20.0, 20.0]], [0, 0])
    s.masses = np.array([18.0])
    m = binding.Model(model, precision)
    got = m.compute(s)
    m.close()
    want = lone_energy(model, 0)
    assert np.abs(got["site_energy"] - want).max() <= 1e-6 * (1 + abs(want))
    assert np.abs(got["force"]).max() <= 1e-6
    assert np.abs(got["virial"]).max() <= 1e-5 and np.abs(got["virial_total"]).max() <= 1e-5
    ref = oracle.compute(model, s)  # the oracle leaves the pair out (r < r_c strictly)
    assert abs(got["energy"] - ref.energy) <= 1e-6 * (1 + abs(ref.energy))


def test_empty_inputs_are_rejected(nep_lib):
    model = two_type_model()
    m = binding.Model(model, "fp32")
    empty = inputs.System(pos=np.zeros((3, 0)), types=np.zeros(0, np.int32), box=np.array([20.0] * 3),
                          pbc=np.array([1, 1, 1], np.int32))
    with pytest.raises(binding.NepError) as e:
        m.compute(empty)
    assert e.value.code == binding.NEP_ERR_ARG
    s = system_of([[1.0, 1.0, 1.0]], [0])
    with pytest.raises(binding.NepError) as e:  # a request without particles
        binding.nep_compute_batch([m.h], np.array([1, 0], np.int32), [0, 0], np.array([[60.0] * 3] * 2),
                                  np.zeros((2, 3), np.int32), s.types, s.pos, np.zeros(2), np.zeros((2, 9)), None,
                                  np.zeros(3), None)
    assert e.value.code == binding.NEP_ERR_ARG
    m.close()


def test_tiny_requests_in_a_batch(nep_lib):
    model = two_type_model()
    m = binding.Model(model, "fp32")
    systems = [system_of([[3.0, 4.0, 5.0]], [1]),
               system_of([[3.0, 4.0, 5.0], [5.0, 4.0, 5.0]], [0, 1]),
               inputs.random_periodic(90, [12.0, 12.0, 12.0], seed=85, min_dist=1.5, n_types=2)]
    req_n, req_box, req_pbc, types, pos = binding.pack_requests(systems)
    n = int(req_n.sum())
    e, wt, F = np.zeros(3), np.zeros((3, 9)), np.zeros(3 * n)
    binding.nep_compute_batch([m.h], req_n, [0, 0, 0], req_box, req_pbc, types, pos, e, wt, None, F, None)
    Fs = binding.unpack_blocks(F, req_n, 3)
    for r, s in enumerate(systems):
        alone = m.compute(s)
        assert e[r] == alone["energy"]
        np.testing.assert_array_equal(Fs[r], alone["force"])
    assert e[0] == pytest.approx(lone_energy(model, 1), rel=1e-6)
    m.close()
