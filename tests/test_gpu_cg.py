"""Coarse-grained mapping on the GPU (nep_cg_map) against the oracle (Eq. 9, 12,
14), host and device memory, accumulation over frames."""
import numpy as np
import pytest

import oracle
from paper_2603_01234_gb300 import binding, inputs
from tests.gpu_common import water_model

pytestmark = pytest.mark.gpu


def atomistic(seed=6):
    model = inputs.random_model(seed=3, rc_radial=5.0, rc_angular=4.0)
    s = inputs.random_periodic(240, [18.0, 19.0, 20.0], seed=seed, min_dist=1.3)
    r = oracle.compute(model, s)
    rng = np.random.default_rng(seed)
    sizes = rng.integers(1, 7, size=80)
    sizes = sizes[np.cumsum(sizes) <= s.n]
    start = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    atoms = rng.permutation(s.n)[:start[-1]].astype(np.int32)
    mass = rng.uniform(1.0, 20.0, size=s.n)
    return s, r, start, atoms, mass


def test_cg_map_matches_oracle_host_and_device(nep_lib):
    import torch
    s, r, start, atoms, mass = atomistic()
    want = oracle.cg_map(start, atoms, mass, s.pos, s.box, s.pbc, r.force, r.virial)
    m = binding.Model(water_model(), "fp64")
    got = binding.nep_cg_map(m.h, start, atoms, mass, s.pos, s.box, s.pbc, r.force, r.virial)
    for g, w in zip(got, want):
        np.testing.assert_allclose(g, w, atol=1e-12)
    dev = torch.device("cuda:0")
    t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa: E731
    n_cg = start.size - 1
    bp = torch.zeros(3, n_cg, dtype=torch.float64, device=dev)
    bf = torch.zeros(3, n_cg, dtype=torch.float64, device=dev)
    bw = torch.zeros(9, n_cg, dtype=torch.float64, device=dev)
    binding.nep_cg_map(m.h, t(start, torch.int32), t(atoms, torch.int32), t(mass), t(s.pos), s.box, s.pbc, t(r.force),
                       t(r.virial), bead_pos=bp, bead_force=bf, bead_virial=bw)
    torch.cuda.synchronize()
    for g, w in zip((bp, bf, bw), want):
        np.testing.assert_allclose(g.cpu().numpy(), w, atol=1e-12)
    m.close()


def test_cg_map_accumulates_time_averages(nep_lib):
    s, r, start, atoms, mass = atomistic(seed=7)
    m = binding.Model(water_model(), "fp64")
    n_cg = start.size - 1
    acc_f, acc_w = np.zeros((3, n_cg)), np.zeros((9, n_cg))
    frames = [(r.force * k, r.virial * (1 + k)) for k in range(1, 4)]
    for f, w in frames:
        binding.nep_cg_map(m.h, start, atoms, mass, s.pos, s.box, s.pbc, f, w, accumulate=True, bead_force=acc_f,
                           bead_virial=acc_w)
    _, bf, bw = oracle.cg_map(start, atoms, mass, s.pos, s.box, s.pbc, r.force, r.virial)
    np.testing.assert_allclose(acc_f / 3, bf * 2.0, atol=1e-12)  # mean of 1, 2, 3 times
    np.testing.assert_allclose(acc_w / 3, bw * 3.0, atol=1e-12)  # mean of 2, 3, 4 times
    m.close()
