"""Batched evaluation (nep_compute_batch) through the C ABI: a batch of mixed
configurations and models gives, for every request, the result of evaluating that
request alone, and matches the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2603_01234_gb300 import binding, inputs
from tests.gpu_common import assert_parity, monolayer_model, small_systems, water_model

pytestmark = pytest.mark.gpu


def mixed_requests(k=12, seed=31):
    rng = np.random.default_rng(seed)
    reqs = []
    for r in range(k):
        n = int(rng.integers(40, 700))
        if r % 2 == 0:
            s = inputs.water_box(n, seed=seed + r)
            reqs.append((0, s))
        else:
            s = inputs.monolayer(int(rng.integers(2, 6)), int(rng.integers(2, 6)), seed=seed + r)
            reqs.append((1, s))
    return reqs


def run_batch(handles, reqs):
    systems = [s for _, s in reqs]
    req_n, req_box, req_pbc, types, pos = binding.pack_requests(systems)
    n = int(req_n.sum())
    e = np.zeros(len(reqs))
    wt = np.zeros((len(reqs), 9))
    U = np.zeros(n)
    F = np.zeros(3 * n)
    W = np.zeros(9 * n)
    binding.nep_compute_batch(handles, req_n, [m for m, _ in reqs], req_box, req_pbc, types, pos, e, wt, U, F, W)
    out = []
    o = 0
    Fs = binding.unpack_blocks(F, req_n, 3)
    Ws = binding.unpack_blocks(W, req_n, 9)
    for r, nr in enumerate(req_n):
        out.append({"energy": e[r], "virial_total": wt[r], "site_energy": U[o:o + nr], "force": Fs[r],
                    "virial": Ws[r]})
        o += nr
    return out


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_equals_alone(nep_lib, precision):
    models = [water_model(), monolayer_model()]
    handles = [binding.Model(p, precision) for p in models]
    reqs = mixed_requests()
    got = run_batch([h.h for h in handles], reqs)
    for (mi, s), g in zip(reqs, got):
        alone = handles[mi].compute(s)
        assert g["energy"] == alone["energy"]
        np.testing.assert_array_equal(g["force"], alone["force"])
        np.testing.assert_array_equal(g["virial"], alone["virial"])
        np.testing.assert_array_equal(g["site_energy"], alone["site_energy"])
        np.testing.assert_array_equal(g["virial_total"], alone["virial_total"])
    for h in handles:
        h.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_matches_oracle(nep_lib, precision):
    models = [water_model(), monolayer_model()]
    handles = [binding.Model(p, precision) for p in models]
    reqs = mixed_requests(k=6, seed=41)
    got = run_batch([h.h for h in handles], reqs)
    for (mi, s), g in zip(reqs, got):
        assert_parity(g, oracle.compute(models[mi], s), precision)
    for h in handles:
        h.close()


def test_batch_device_equals_host(nep_lib):
    import torch
    models = [water_model(), monolayer_model()]
    handles = [binding.Model(p, "fp32") for p in models]
    reqs = mixed_requests(k=8, seed=51)
    host = run_batch([h.h for h in handles], reqs)
    systems = [s for _, s in reqs]
    req_n, req_box, req_pbc, types, pos = binding.pack_requests(systems)
    dev = torch.device("cuda:0")
    n = int(req_n.sum())
    t = torch.from_numpy(types).to(dev)
    P = torch.from_numpy(pos).to(dev)
    e = torch.zeros(len(reqs), dtype=torch.float64, device=dev)
    wt = torch.zeros(len(reqs), 9, dtype=torch.float64, device=dev)
    F = torch.zeros(3 * n, dtype=torch.float64, device=dev)
    binding.nep_compute_batch([h.h for h in handles], req_n, [m for m, _ in reqs], req_box, req_pbc, t, P, e, wt,
                              None, F, None)
    torch.cuda.synchronize()
    Fs = binding.unpack_blocks(F.cpu().numpy(), req_n, 3)
    for r in range(len(reqs)):
        assert float(e[r]) == host[r]["energy"]
        np.testing.assert_array_equal(wt[r].cpu().numpy(), host[r]["virial_total"])
        np.testing.assert_array_equal(Fs[r], host[r]["force"])
    for h in handles:
        h.close()


def test_batch_rejects_mismatched_models(nep_lib):
    a = binding.Model(water_model(), "fp32")
    b = binding.Model(water_model(), "fp64")
    s = inputs.water_box(100, seed=3)
    req_n, req_box, req_pbc, types, pos = binding.pack_requests([s, s])
    with pytest.raises(binding.NepError) as e:
        binding.nep_compute_batch([a.h, b.h], req_n, [0, 1], req_box, req_pbc, types, pos, np.zeros(2))
    assert e.value.code == binding.NEP_ERR_ARG
    a.close()
    b.close()


def test_batches_of_one_size_class_share_a_graph(nep_lib):
    """Consecutive batches whose sizes fall in one size class replay one captured
    graph (the kernels read the batch's sizes from the device); every request of
    every batch still equals its evaluation alone, bitwise.  The batches differ in
    their number of requests, so the tables' offsets would differ if they were laid
    out by count rather than by capacity."""
    models = [water_model(), monolayer_model()]
    batch_handles = [binding.Model(p, "fp32") for p in models]
    alone_handles = [binding.Model(p, "fp32") for p in models]
    rng = np.random.default_rng(71)
    for b in range(6):
        k = int(rng.integers(3, 9))
        reqs = []
        for r in range(k):
            n = int(rng.integers(80, 160))
            reqs.append((0, inputs.water_box(n, seed=1000 * b + r)) if r % 2 == 0 else
                        (1, inputs.monolayer(3, 2, seed=1000 * b + r)))
        got = run_batch([h.h for h in batch_handles], reqs)
        for (mi, s), g in zip(reqs, got):
            alone = alone_handles[mi].compute(s)
            assert g["energy"] == alone["energy"]
            np.testing.assert_array_equal(g["force"], alone["force"])
            np.testing.assert_array_equal(g["virial"], alone["virial"])
    for h in batch_handles + alone_handles:
        h.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_small_and_large_batches_build_the_same_lists(nep_lib, precision):
    """A configuration evaluated alone (a small batch: the warp-per-particle
    neighbour kernel) and inside a batch of more than 96 work items (the
    thread-per-particle kernel) gives bitwise equal results: both kernels write the
    same neighbour lists in the same order."""
    models = [water_model(), monolayer_model()]
    handles = [binding.Model(p, precision) for p in models]
    small = [(0, inputs.water_box(900, seed=71)), (1, inputs.monolayer(4, 3, seed=72))]
    big = (0, inputs.water_box(20000, seed=73))  # 157 work items on its own
    got = run_batch([h.h for h in handles], small + [big])
    for (mi, s), g in zip(small, got):
        alone = handles[mi].compute(s)
        assert g["energy"] == alone["energy"]
        np.testing.assert_array_equal(g["force"], alone["force"])
        np.testing.assert_array_equal(g["virial"], alone["virial"])
    for h in handles:
        h.close()


@pytest.mark.parametrize("case", [c for c in small_systems()], ids=[c[0] for c in small_systems()])
def test_thread_and_warp_neighbour_kernels_agree_on_small_systems(nep_lib, case):
    """Every small parity case (tiny boxes whose stencils repeat cells as images,
    open axes, several types, the second compiled shape) evaluated alone (a small
    batch: the warp-per-particle neighbour kernel) equals the same configuration
    inside a batch of copies spanning more than 96 work items (the thread-per-
    particle kernel), bitwise."""
    name, model, system = case
    h = binding.Model(model, "fp32")
    copies = -(-97 // -(-system.n // 128))  # enough copies for more than 96 work items
    got = run_batch([h.h], [(0, system)] * copies)
    alone = h.compute(system)
    for g in (got[0], got[-1]):
        assert g["energy"] == alone["energy"]
        np.testing.assert_array_equal(g["force"], alone["force"])
        np.testing.assert_array_equal(g["virial"], alone["virial"])
    h.close()
