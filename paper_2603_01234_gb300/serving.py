"""Continuous-batching server of energy / force / virial requests.

Requests (a model index and a configuration) arrive over time.  `lanes` worker
threads each own a set of model handles -- and therefore a device workspace -- and
repeatedly admit the requests that have arrived, in arrival order, until the
lane's memory budget is reached, then evaluate them with one nep_compute_batch
call.  The call releases the GIL, so while one lane's batch runs on the GPU the
other lanes admit the requests that arrived meanwhile and launch their own
batches: work of different batches overlaps on the device, and a request never
waits for a batch that is already running.

Admission is by memory: every request carries the device workspace bytes the
library reports for it (nep_request_workspace: particle arrays, neighbour lists at
the handle's capacities, cells, work items), and a lane admits requests while their
sum stays within its budget (less the 1/8 by which a batch's size classes may round
up).  Each lane packs its batches into page-locked host buffers, so the copies to
and from the device run at link speed.

With lanes=1 and max_requests=1 the same server evaluates one request per launch
sequence (the plain, unbatched form).

With device_resident=True the requests' configurations live on the GPU (types and
positions as torch CUDA tensors) and so do the results: each lane concatenates its
batch on its own CUDA stream and evaluates it there, and no request data crosses
the host link.
"""
from __future__ import annotations

import threading
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import binding

# a batch's capacities round up to size classes: at most 9/8 of the sum over requests
CLASS_MARGIN = 9.0 / 8.0


@dataclass
class Request:
    rid: int
    model: int
    system: object
    arrival: float = 0.0
    done: float = 0.0
    result: dict | None = None
    batch_size: int = 0
    ws: int = 0  # device workspace bytes this request adds to a batch


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


class Staging:
    """One lane's host buffers for a batch (inputs and outputs), grown as needed:
    page-locked (nep_host_alloc) or, with pinned=False, ordinary numpy memory."""

    # bytes per particle: types int32, positions 3 f64, forces 3 f64, virials 9 f64
    _LAYOUT = (("types", 4, 1, np.int32), ("pos", 8, 3, np.float64), ("force", 8, 3, np.float64),
               ("virial", 8, 9, np.float64))

    def __init__(self, pinned=True):
        self.pinned = pinned
        self.n_cap = 0
        self.k_cap = 0
        self.buf = None
        self.arrays = {}

    def ensure(self, n, k):
        if n <= self.n_cap and k <= self.k_cap:
            return self.arrays
        self.close()
        self.n_cap = max(n, int(self.n_cap * 1.25))
        self.k_cap = max(k, int(self.k_cap * 1.25))
        sizes = [(name, w * self.n_cap, dt) for name, _, w, dt in self._LAYOUT]
        sizes += [("energy", self.k_cap, np.float64), ("virial_total", 9 * self.k_cap, np.float64)]
        if self.pinned:
            total = sum(((c * np.dtype(dt).itemsize + 255) // 256) * 256 for _, c, dt in sizes)
            self.buf = binding.PinnedBuffer(total)
            off = 0
            for name, c, dt in sizes:
                self.arrays[name] = self.buf.view(off, c, dt)
                off += ((c * np.dtype(dt).itemsize + 255) // 256) * 256
        else:
            self.arrays = {name: np.zeros(c, dt) for name, c, dt in sizes}
        return self.arrays

    def close(self):
        self.arrays = {}
        if self.buf is not None:
            self.buf.close()
            self.buf = None


class Server:
    def __init__(self, params_list, precision="fp32", lanes=2, lane_bytes=2 << 30, max_requests=4096, device=0,
                 keep_results=True, pinned=True, device_resident=False):
        self.params_list = params_list
        self.device = device
        self.device_resident = device_resident
        self.lanes = []
        for _ in range(lanes):
            self.lanes.append([binding.Model(p, precision, device) for p in params_list])
        # admission budget: the lane's bytes less the size classes' rounding
        self.max_bytes = max(1, int(lane_bytes / CLASS_MARGIN))
        self.max_requests = max_requests
        self.keep_results = keep_results
        self.pinned = pinned
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

    def workspace_bytes(self, r):
        """Device workspace the request adds to a batch, as the library reports it
        for the lane workspace (models[0] of a lane) that would evaluate it."""
        return binding.nep_request_workspace([m.h for m in self.lanes[0]], r.model, r.system.n, r.system.box,
                                             r.system.pbc)

    # -- admission --------------------------------------------------------------
    def _admit(self):
        """Take arrived requests in order until the memory or request budget; a
        request larger than the whole budget goes alone."""
        batch, used = [], 0
        while self._pending and len(batch) < self.max_requests:
            r = self._pending[0]
            if batch and used + r.ws > self.max_bytes:
                break
            batch.append(self._pending.popleft())
            used += r.ws
        return batch

    def _lane(self, handles):
        hs = [m.h for m in handles]
        staging = None if self.device_resident else Staging(self.pinned)
        stream = None
        if self.device_resident:
            import torch
            stream = torch.cuda.Stream(device=self.device)
        try:
            while True:
                with self._cv:
                    while not self._pending and not self._closed:
                        self._cv.wait()
                    if not self._pending and self._closed:
                        return
                    batch = self._admit()
                if self.device_resident:
                    self._run_batch_device(hs, batch, stream)
                else:
                    self._run_batch(hs, batch, staging)
        finally:
            if staging is not None:
                staging.close()

    def _run_batch_device(self, hs, batch, stream):
        """A batch of device-resident requests: concatenated on the lane's stream,
        evaluated there (the call synchronises once), results kept as device views."""
        import torch

        k = len(batch)
        req_n = np.array([r.system.n for r in batch], np.int32)
        n = int(req_n.sum())
        req_box = np.array([r.system.box for r in batch], np.float64)
        req_pbc = np.array([r.system.pbc for r in batch], np.int32)
        dev = torch.device("cuda", self.device)
        with torch.cuda.stream(stream):
            types = torch.cat([r.system.types for r in batch])
            pos = torch.cat([r.system.pos.reshape(-1) for r in batch])
            e = torch.empty(k, dtype=torch.float64, device=dev)
            wt = torch.empty(9 * k, dtype=torch.float64, device=dev)
            F = torch.empty(3 * n, dtype=torch.float64, device=dev)
            W = torch.empty(9 * n, dtype=torch.float64, device=dev) if self.keep_results else None
            binding.nep_compute_batch(hs, req_n, [r.model for r in batch], req_box, req_pbc, types, pos, e, wt, None,
                                      F, W, stream=stream.cuda_stream)
        t = time.perf_counter()
        o = 0
        for q, r in enumerate(batch):
            r.done = t
            r.batch_size = k
            if self.keep_results:
                nr = r.system.n
                r.result = {"energy": e[q], "virial_total": wt[9 * q:9 * q + 9], "force": F[3 * o:3 * (o + nr)].view(3, nr),
                            "virial": W[9 * o:9 * (o + nr)].view(9, nr)}
                o += nr
        with self._cv:
            self.batches += 1
            self.batch_requests += k

    def _run_batch(self, hs, batch, staging):
        k = len(batch)
        req_n = np.array([r.system.n for r in batch], np.int32)
        n = int(req_n.sum())
        req_box = np.array([r.system.box for r in batch], np.float64)
        req_pbc = np.array([r.system.pbc for r in batch], np.int32)
        a = staging.ensure(n, k)
        types, pos = a["types"][:n], a["pos"][:3 * n]
        o = 0
        for r in batch:  # pack straight into the staging buffers
            nr = r.system.n
            types[o:o + nr] = r.system.types
            pos[3 * o:3 * (o + nr)] = np.asarray(r.system.pos, np.float64).reshape(-1)
            o += nr
        e, wt = a["energy"][:k], a["virial_total"][:9 * k].reshape(k, 9)
        F = a["force"][:3 * n]
        W = a["virial"][:9 * n] if self.keep_results else None
        binding.nep_compute_batch(hs, req_n, [r.model for r in batch], req_box, req_pbc, types, pos, e, wt, None, F,
                                  W)
        t = time.perf_counter()
        if self.keep_results:
            Fs = binding.unpack_blocks(F, req_n, 3)
            Ws = binding.unpack_blocks(W, req_n, 9)
        for q, r in enumerate(batch):
            r.done = t
            r.batch_size = k
            if self.keep_results:
                r.result = {"energy": float(e[q]), "virial_total": wt[q].copy(), "force": Fs[q].copy(),
                            "virial": Ws[q].copy()}
        with self._cv:
            self.batches += 1
            self.batch_requests += k

    # -- driving ------------------------------------------------------------------
    def serve(self, requests, arrival_times):
        """Release request k at arrival_times[k] seconds after the start (sorted),
        serve all of them, return ServeStats."""
        reqs = list(requests)
        for r in reqs:
            if not r.ws:
                r.ws = self.workspace_bytes(r)
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
