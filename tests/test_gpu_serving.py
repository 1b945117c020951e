"""Continuous-batching server: every served result equals the result of evaluating
the request alone, requests arriving while batches run are admitted, and batches
of different lanes overlap."""
import numpy as np
import pytest

from paper_2603_01234_gb300 import binding, inputs, serving
from tests.gpu_common import monolayer_model, water_model

pytestmark = pytest.mark.gpu


def test_served_results_equal_alone(nep_lib):
    models = [water_model(), monolayer_model()]
    stream = inputs.request_stream(n_requests=120, seed=61, n_min=64, n_max=1024)
    reqs = [serving.Request(k, m, s) for k, (m, s) in enumerate(stream)]
    srv = serving.Server(models, "fp32", lanes=2, lane_bytes=64 << 20)
    arrivals = serving.poisson_arrivals(len(reqs), rate=4000.0, seed=62)
    st = srv.serve(reqs, arrivals)
    assert st.n_requests == len(reqs) and np.all(st.latencies_s > 0)
    assert st.batches < len(reqs)  # requests were batched
    alone = [binding.Model(p, "fp32") for p in models]
    for r in reqs:
        ref = alone[r.model].compute(r.system)
        assert r.result["energy"] == ref["energy"]
        np.testing.assert_array_equal(r.result["force"], ref["force"])
        np.testing.assert_array_equal(r.result["virial"], ref["virial"])
    for m in alone:
        m.close()
    srv.close()


def test_device_resident_serving_equals_alone(nep_lib):
    """Requests whose configurations are CUDA tensors are served without host
    copies; every result (a device tensor) equals the request evaluated alone."""
    torch = pytest.importorskip("torch")
    models = [water_model(), monolayer_model()]
    stream = inputs.request_stream(n_requests=60, seed=64, n_min=64, n_max=1024)
    dev = torch.device("cuda", 0)
    reqs = []
    for k, (m, s) in enumerate(stream):
        ds = inputs.System(pos=torch.from_numpy(np.ascontiguousarray(s.pos)).to(dev),
                           types=torch.from_numpy(s.types.astype(np.int32)).to(dev), box=s.box, pbc=s.pbc)
        reqs.append(serving.Request(k, m, ds))
    srv = serving.Server(models, "fp32", lanes=2, lane_bytes=64 << 20, device_resident=True)
    st = srv.serve(reqs, serving.poisson_arrivals(len(reqs), rate=4000.0, seed=65))
    assert st.n_requests == len(reqs) and st.batches < len(reqs)
    alone = [binding.Model(p, "fp32") for p in models]
    for r, (m, s) in zip(reqs, stream):
        ref = alone[m].compute(s)
        assert float(r.result["energy"]) == ref["energy"]
        np.testing.assert_array_equal(r.result["force"].cpu().numpy(), ref["force"])
        np.testing.assert_array_equal(r.result["virial"].cpu().numpy(), ref["virial"])
    for m in alone:
        m.close()
    srv.close()


def test_memory_admission_bounds_batches(nep_lib):
    models = [water_model(), monolayer_model()]
    stream = inputs.request_stream(n_requests=40, seed=63, n_min=200, n_max=800)
    reqs = [serving.Request(k, m, s) for k, (m, s) in enumerate(stream)]
    srv = serving.Server(models, "fp32", lanes=1, lane_bytes=6 << 20)
    cap = srv.max_bytes
    seen = []
    orig = srv._run_batch

    def spy(hs, batch, staging):
        seen.append((sum(r.ws for r in batch), len(batch)))
        orig(hs, batch, staging)
    srv._run_batch = spy
    srv.serve(reqs, np.zeros(len(reqs)))
    assert sum(k for _, k in seen) == len(reqs)
    assert all(r.ws > 0 for r in reqs)
    assert all(used <= cap or k == 1 for used, k in seen)
    assert any(k > 1 for _, k in seen) and len(seen) > 1
    srv.close()


def test_reported_workspace_bounds_the_allocation(nep_lib):
    """What a fresh handle allocates for a batch stays within 9/8 of the sum of
    nep_request_workspace over its requests (list capacities fixed beforehand, so
    that the query and the batch use the same)."""
    models = [water_model(), monolayer_model()]
    stream = inputs.request_stream(n_requests=60, seed=64, n_min=200, n_max=3000)
    handles = [binding.Model(p, "fp32") for p in models]
    binding.nep_set_capacity(handles[0].h, 160, 64)
    hs = [h.h for h in handles]
    systems = [s for _, s in stream]
    ws = sum(binding.nep_request_workspace(hs, mi, s.n, s.box, s.pbc) for mi, s in stream)
    req_n, req_box, req_pbc, types, pos = binding.pack_requests(systems)
    n = int(req_n.sum())
    k = len(systems)
    binding.nep_compute_batch(hs, req_n, [m for m, _ in stream], req_box, req_pbc, types, pos, np.zeros(k),
                              np.zeros((k, 9)), None, np.zeros(3 * n), np.zeros(9 * n))
    assert binding.nep_get_capacity(handles[0].h) == (160, 64)  # no overflow regrowth in between
    used = binding.nep_workspace_bytes(handles[0].h)
    assert 0.5 * ws < used <= serving.CLASS_MARGIN * ws + 65536, (used, ws)
    for h in handles:
        h.close()
