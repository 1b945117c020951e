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


def test_memory_admission_bounds_batches(nep_lib):
    models = [water_model(), monolayer_model()]
    stream = inputs.request_stream(n_requests=40, seed=63, n_min=200, n_max=800)
    reqs = [serving.Request(k, m, s) for k, (m, s) in enumerate(stream)]
    srv = serving.Server(models, "fp32", lanes=1, lane_bytes=2 << 20)
    cap = srv.max_particles
    seen = []
    orig = srv._run_batch

    def spy(hs, batch):
        seen.append((sum(r.system.n for r in batch), len(batch)))
        orig(hs, batch)
    srv._run_batch = spy
    srv.serve(reqs, np.zeros(len(reqs)))
    assert sum(k for _, k in seen) == len(reqs)
    assert all(beads <= cap or k == 1 for beads, k in seen)
    assert any(k > 1 for _, k in seen)
    srv.close()
