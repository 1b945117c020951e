"""Host logic of the continuous-batching server (paper_2603_01234_gb300/serving.py)
without a GPU: admission order and budgets (by each request's workspace bytes), and
the threaded serve loop with the batched evaluation and the workspace query replaced
by host stubs that write per-request values, so that packing into the lane's
staging buffers, unpacking and hand-back of results to their requests are checked."""
import threading

import numpy as np
import pytest

from paper_2603_01234_gb300 import binding, inputs, serving


def make_requests(sizes, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for k, n in enumerate(sizes):
        s = inputs.System(pos=rng.uniform(0.0, 10.0, (3, n)), types=np.zeros(n, np.int32),
                          box=np.array([10.0, 10.0, 10.0]), pbc=np.array([1, 1, 1], np.int32))
        out.append(serving.Request(rid=k, model=k % 2, system=s, ws=n))  # one byte per particle
    return out


def bare_server(max_bytes, max_requests):
    srv = serving.Server.__new__(serving.Server)  # no model handles (they need a GPU)
    srv.max_bytes = max_bytes
    srv.max_requests = max_requests
    srv.keep_results = True
    srv._cv = threading.Condition()
    from collections import deque
    srv._pending = deque()
    srv._closed = False
    srv.batches = srv.batch_requests = 0
    return srv


def test_admission_in_arrival_order_within_budgets():
    srv = bare_server(max_bytes=100, max_requests=3)
    reqs = make_requests([40, 50, 20, 10, 300, 5])
    srv._pending.extend(reqs)
    assert [r.rid for r in srv._admit()] == [0, 1]        # 40 + 50; adding 20 would pass 100
    assert [r.rid for r in srv._admit()] == [2, 3]        # 20 + 10; 300 does not fit
    assert [r.rid for r in srv._admit()] == [4]           # an oversized request goes alone
    assert [r.rid for r in srv._admit()] == [5]
    assert srv._admit() == []
    srv2 = bare_server(max_bytes=10_000, max_requests=2)
    srv2._pending.extend(make_requests([1, 1, 1, 1, 1]))
    assert [len(srv2._admit()) for _ in range(3)] == [2, 2, 1]  # request budget


def test_serve_loop_hands_each_result_to_its_request(monkeypatch):
    calls = []

    class FakeModel:
        def __init__(self, params, precision="fp32", device=0):
            self.h = object()

        def close(self):
            pass

    def fake_batch(handles, req_n, req_model, req_box, req_pbc, types, pos, energy, virial_total, site, force,
                   virial):
        calls.append(len(req_n))
        o = 0
        for r, n in enumerate(req_n):
            block = pos[3 * o:3 * (o + n)].reshape(3, n)
            energy[r] = n + 1000 * req_model[r]            # identifies the request and its model
            virial_total[r] = block.sum()
            force[3 * o:3 * (o + n)] = -block.reshape(-1)  # identifies every particle
            if virial is not None:
                virial[9 * o:9 * (o + n)] = r
            o += n

    monkeypatch.setattr(binding, "Model", FakeModel)
    monkeypatch.setattr(binding, "nep_compute_batch", fake_batch)
    monkeypatch.setattr(binding, "nep_request_workspace", lambda hs, model, n, box, pbc: 10 * n)
    params = [inputs.random_model(seed=1), inputs.random_model(seed=2)]
    srv = serving.Server(params, lanes=3, lane_bytes=2250 * 9 // 8 + 1, max_requests=8, pinned=False)
    assert srv.max_bytes == 2250
    sizes = [64, 17, 130, 5, 99, 64, 1, 250, 33, 70]
    reqs = make_requests(sizes, seed=3)
    stats = srv.serve(reqs, serving.poisson_arrivals(len(reqs), rate=2000.0, seed=4))
    srv.close()
    assert stats.n_requests == len(reqs) and stats.n_particles == sum(sizes)
    assert sum(calls) == len(reqs) and stats.batches == len(calls)
    assert np.all(stats.latencies_s >= 0.0) and stats.throughput > 0
    for r in reqs:
        assert r.result["energy"] == r.system.n + 1000 * r.model
        np.testing.assert_array_equal(r.result["force"], -r.system.pos)
        assert r.result["virial_total"] == pytest.approx(r.system.pos.sum())
        assert r.result["force"].shape == (3, r.system.n) and r.result["virial"].shape == (9, r.system.n)
        assert 1 <= r.batch_size <= 8
