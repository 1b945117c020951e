"""Continuous-batching server of energy / force / virial requests.

Requests (a model index and a configuration) arrive over time.  `lanes` worker
threads each own a set of model handles -- and therefore a device workspace -- and
repeatedly admit the requests that have arrived, in arrival order, until the
batch's particle budget is reached, then evaluate them with one nep_compute_batch
call.  The call releases the GIL, so while one lane's batch runs on the GPU another
lane admits the requests that arrived meanwhile and launches its own batch: work of
different batches overlaps on the device, and a request never waits for a batch
that is already running.  Admission is by memory: the particle budget per batch is
derived from a byte budget per lane and the workspace bytes a particle needs.

With lanes=1 and max_requests=1 the same server evaluates one request per launch
sequence (the plain, unbatched form).
"""
from __future__ import annotations

import threading
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import binding


# Device workspace bytes per particle of a batch (FP32 form): cell-relative records,
# neighbour lists at their usual capacity, radial and angular gradients, outputs.
def bytes_per_particle(params, list_capacity=160):
    rs = 4
    return (2 * 16 + 6 * 4 + 4 * list_capacity + rs * (1 + params.n_types * 8 + 24 * params.n_desc_angular)
            + 8 * (1 + 3 + 9) + 8 * 4)


@dataclass
class Request:
    rid: int
    model: int
    system: object
    arrival: float = 0.0
    done: float = 0.0
    result: dict | None = None
    batch_size: int = 0


@dataclass
class ServeStats:
    n_requests: int
    n_particles: int
    wall_s: float
    latencies_s: np.ndarray
    batches: int
    mean_batch_requests: float
    extra: dict = field(default_factory=dict)

    @property
    def throughput(self):
        """Particle evaluations per second over the whole run."""
        return self.n_particles / self.wall_s

    def pct(self, q):
        return float(np.percentile(self.latencies_s, q))


class Server:
    def __init__(self, params_list, precision="fp32", lanes=2, lane_bytes=2 << 30, max_requests=4096, device=0,
                 keep_results=True):
        self.params_list = params_list
        self.lanes = []
        for _ in range(lanes):
            self.lanes.append([binding.Model(p, precision, device) for p in params_list])
        bpp = max(bytes_per_particle(p) for p in params_list)
        self.max_particles = max(1, int(lane_bytes // bpp))
        self.max_requests = max_requests
        self.keep_results = keep_results
        self._cv = threading.Condition()
        self._pending = deque()
        self._closed = False
        self.batches = 0
        self.batch_requests = 0

    def close(self):
        for lane in self.lanes:
            for m in lane:
                m.close()
        self.lanes = []

    # -- admission --------------------------------------------------------------
    def _admit(self):
        """Take arrived requests in order until the particle or request budget."""
        batch, beads = [], 0
        while self._pending and len(batch) < self.max_requests:
            r = self._pending[0]
            if batch and beads + r.system.n > self.max_particles:
                break
            batch.append(self._pending.popleft())
            beads += r.system.n
        return batch

    def _lane(self, handles):
        hs = [m.h for m in handles]
        while True:
            with self._cv:
                while not self._pending and not self._closed:
                    self._cv.wait()
                if not self._pending and self._closed:
                    return
                batch = self._admit()
            self._run_batch(hs, batch)

    def _run_batch(self, hs, batch):
        systems = [r.system for r in batch]
        req_n, req_box, req_pbc, types, pos = binding.pack_requests(systems)
        n = int(req_n.sum())
        k = len(batch)
        e = np.zeros(k)
        wt = np.zeros((k, 9))
        F = np.zeros(3 * n)
        W = np.zeros(9 * n) if self.keep_results else None
        binding.nep_compute_batch(hs, req_n, [r.model for r in batch], req_box, req_pbc, types, pos, e, wt, None, F, W)
        t = time.perf_counter()
        if self.keep_results:
            Fs = binding.unpack_blocks(F, req_n, 3)
            Ws = binding.unpack_blocks(W, req_n, 9)
        for q, r in enumerate(batch):
            r.done = t
            r.batch_size = k
            if self.keep_results:
                r.result = {"energy": e[q], "virial_total": wt[q], "force": Fs[q], "virial": Ws[q]}
        with self._cv:
            self.batches += 1
            self.batch_requests += k

    # -- driving ------------------------------------------------------------------
    def serve(self, requests, arrival_times):
        """Release request k at arrival_times[k] seconds after the start (sorted),
        serve all of them, return ServeStats."""
        reqs = list(requests)
        self._closed = False
        self.batches = self.batch_requests = 0
        threads = [threading.Thread(target=self._lane, args=(lane,), daemon=True) for lane in self.lanes]
        for th in threads:
            th.start()
        t0 = time.perf_counter()
        for r, at in zip(reqs, arrival_times):
            now = time.perf_counter() - t0
            if at > now:
                time.sleep(at - now)
            r.arrival = time.perf_counter()
            with self._cv:
                self._pending.append(r)
                self._cv.notify()
        with self._cv:
            self._closed = True
            self._cv.notify_all()
        for th in threads:
            th.join()
        wall = max(r.done for r in reqs) - t0
        lat = np.array([r.done - r.arrival for r in reqs])
        return ServeStats(len(reqs), sum(r.system.n for r in reqs), wall, lat, self.batches,
                          self.batch_requests / max(1, self.batches))


def poisson_arrivals(n, rate, seed):
    """Arrival times (s) of a Poisson process of `rate` requests/s."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))
