#!/usr/bin/env python
"""Benchmark of the NEP MD step (cell list -> neighbours -> descriptors -> network ->
forces + virials -> FP64 reductions -> velocity-Verlet) on the 100,000-bead CG water
system, reported as bead-steps/s and ns/day.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one velocity-Verlet step of the whole system.  Timed region: K steps, each
one library call that replays the step's captured CUDA graph, bracketed by CUDA events
on the launch stream, with a 256 MiB write between steps to flush the 126 MB L2 (the
step's working set is smaller than L2).  Inputs are resident in HBM before timing.
Per-stage times come from a second pass of K steps launched eagerly with CUDA events
between the stages.  With N > 1 (torchrun) every rank runs an independent
replica (the method shards by independent systems; no collective on the data path);
value = all ranks' bead-steps / the slowest rank's time.

--impl reference times the FP64 CPU oracle (test infrastructure) on a bounded sample
of the same workload on this host's cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2603_01234_gb300 import inputs  # noqa: E402

METRIC = "bead-steps/s (100k-bead CG water MD step)"
UNIT = "bead-steps/s"
DT_FS = 10.0
FLOPS_PEAK_NOTE = "FP32 ALU peak = SMs (device-reported) x 128 FP32 lanes x 2 flop/FMA x clock"

# DRAM bytes per particle of one launch of the dominant kernel, from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum); valid only for the evaluate.cu
# source it was taken on, otherwise the bench reports traffic as null.
KERNEL_TRAFFIC = {"evaluate_cu_sha1": "d2c4d44fa96296386a005caeb16897c4dc11cf15", "bytes_per_particle": 454.2,
                  "kernel": "descriptor_network",
                  "capture": "ncu --set full, k_descriptor (descriptor + network + angular forces), 100,000-bead water, "
                             "variants 3,3,4, cold caches: 45.31 MB read + 0.11 MB written per launch"}


N_BEADS = 100_000
WORKLOAD = "water100k"

# name -> (description, dt in fs)
WORKLOADS = {
    "water100k": ("CG water, 1 type, density 0.0334/A^3, periodic cube", 10.0),
    "water512": ("CG water, 512 beads (8^3 lattice, 3.1 A), periodic cube 24.8 A", 10.0),
    "monolayer200k": ("4-type distorted hexagonal monolayer, 250x200 cells, periodic x,y, open z", 20.0),
    "nanowire1M": ("atom-and-bead nanowire: FCC core r=15 A (type 0) in 2 bead sheaths, periodic x", 5.0),
}


def workload(name=None):
    """(model, system, velocities) of a named workload; seeds fixed."""
    name = name or WORKLOAD
    if name == "water100k":
        model = inputs.random_model(n_types=1, n_desc_radial=5, n_desc_angular=4, n_basis_radial=8,
                                    n_basis_angular=8, l_max=4, hidden=30, rc_radial=8.0, rc_angular=5.0, seed=1)
        system = inputs.water_box(N_BEADS, density=0.0334, seed=1001)
        system.masses = np.array([18.0])
    elif name == "water512":
        model = inputs.random_model(n_types=1, hidden=30, rc_radial=8.0, rc_angular=5.0, seed=1)
        system = inputs.water_small(seed=1000)
    elif name == "monolayer200k":
        model = inputs.random_model(n_types=4, hidden=50, rc_radial=15.0, rc_angular=11.0, seed=2)
        system = inputs.monolayer(250, 200, seed=1002)
    elif name == "nanowire1M":
        model = inputs.random_model(n_types=3, hidden=40, rc_radial=7.0, rc_angular=5.0, seed=4)
        system = inputs.nanowire(1_000_000, seed=1003)
    else:
        raise ValueError(name)
    vel = inputs.maxwell_boltzmann(system, 300.0, seed=7)
    return model, system, vel


def config_dict(system, name=None):
    name = name or WORKLOAD
    m = workload_model_note(name)
    return {"workload": f"{WORKLOADS[name][0]}; {system.n} particles; box "
                        f"{system.box[0]:.1f} x {system.box[1]:.1f} x {system.box[2]:.1f} A",
            "model": m, "n_beads": system.n, "dt_fs": WORKLOADS[name][1],
            "integrator": "velocity-Verlet NVE (FP64)",
            "precision": "FP32 descriptors/network/forces, FP64 reductions+integration",
            "l2": "flushed between timed steps (256 MiB write)",
            "state": "every timed step starts from the same configuration (positions, velocities and forces "
                     "restored before the step, outside the timed events)",
            "data": "synthetic (seeded lattice, Maxwell-Boltzmann 300 K)"}


def workload_model_note(name):
    return {"water100k": "NEP4-form random weights N(0,0.1): n_R=5, n_A=4, K_R=K_A=8, l_max=4, H=30, r_c 8/5 A",
            "water512": "as water100k",
            "monolayer200k": "4 types, H=50, r_c 15/11 A, n_R=5, n_A=4, K=8, l_max=4",
            "nanowire1M": "3 types, H=40, r_c 7/5 A, n_R=5, n_A=4, K=8, l_max=4"}[name]


# ---- algorithmic work per kernel (FMA = 2 flop; sin/cos, rsqrt, tanh, div = 1) ----
def algorithmic_flops(m, pairs_r, pairs_a, n, fused=True):
    """Minimal flops of one evaluation per launch: every ordered pair's gradient
    f_ij counted once (the gather form computes both directions, so it does more),
    and the linear Chebyshev contractions of Eq. 6 moved to the bead level where
    the sums allow it.  basis(K) = 10 + 5 (K - 2) for f_k, basis'(K) = 14 + 11 (K - 2)
    for f_k and f_k'.

    descriptor+network kernel, per
      radial pair   13 (pair vector, r) + basis(K_R) + K_R (sum of f_k)
      angular pair  16 (+ unit vector) + basis(K_A) + 2 n_A K_A (g_n) + 60 (Y_lm, l<=4)
                    + 2 n_A 24 (A_nlm)
      bead          2 T n_R K_R (q_n) + 2 n_A 24 (q_nl) + H (4 N_des + 6) (Eq. 2 and dU/dq)
                    + 2 T n_R K_R (radial gradient in the basis) + 2 n_A 24 (Phi)
    pair forces, per
      radial pair   13 + basis'(K_R) + 2 K_R (f_ij) + 6 (F) + 18 (W)
      angular pair  16 + basis'(K_A) + 4 n_A K_A (g, g') + 150 (Y_lm and grad Y_lm)
                    + 24 (4 n_A + 10) (one direction's contraction) + 12 (F) + 18 (W)
    In the FP32 form the angular pairs' forces run inside the descriptor kernel
    (Phi_i stays in registers) and the radial pairs' in the second kernel.
    """
    nR, nA, KR, KA, H, T = (m.n_desc_radial, m.n_desc_angular, m.n_basis_radial, m.n_basis_angular, m.hidden,
                            m.n_types)
    nd = m.n_des
    basis = lambda K: 10 + 5 * (K - 2)  # noqa: E731
    basis_d = lambda K: 14 + 11 * (K - 2)  # noqa: E731
    d_r = 13 + basis(KR) + KR
    d_a = 16 + basis(KA) + 2 * nA * KA + 60 + 2 * nA * 24
    d_b = 2 * T * nR * KR + 2 * nA * 24 + H * (4 * nd + 6) + 2 * T * nR * KR + 2 * nA * 24
    f_r = 13 + basis_d(KR) + 2 * KR + 6 + 18
    f_a = 16 + basis_d(KA) + 4 * nA * KA + 150 + 24 * (4 * nA + 10) + 12 + 18
    # the FP32 form's two evaluation kernels: descriptor + network + angular pair
    # forces (stage "descriptor_network"), radial pair forces + outputs ("force_virial");
    # the FP64 form (fused=False): descriptor + network, then all pair forces
    if not fused:
        return {"descriptor_network": d_r * pairs_r + d_a * pairs_a + d_b * n,
                "force_virial": f_r * pairs_r + f_a * pairs_a}
    return {"descriptor_network": d_r * pairs_r + d_a * pairs_a + d_b * n + f_a * pairs_a,
            "force_virial": f_r * pairs_r}


# ---- clocks sampler ------------------------------------------------------------
CLOCK_REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


def summarize_clocks(samples, t0=None, t1=None):
    """Clock samples [(host time, nvidia-smi CSV line)] to the bench's clocks record.
    The statistics use the samples taken in [t0, t1] (the timed region); when none
    fell inside it, the nearest sample on each side stands in, and the record says
    so."""
    rows = []
    for t, ln in samples:
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 9:
            continue
        try:
            sm, smax, pw = float(f[1]), float(f[2]), float(f[3])
        except ValueError:
            continue
        act = [name for k, name in enumerate(CLOCK_REASONS) if f[5 + k].lower().startswith("active")]
        rows.append((t, sm, smax, pw, act))
    inside = rows if t0 is None else [r for r in rows if t0 <= r[0] <= t1]
    window = "timed region"
    if not inside and rows:
        before = [r for r in rows if r[0] < t0]
        after = [r for r in rows if r[0] > t1]
        inside = before[-1:] + after[:1]
        window = "nearest samples around the timed region (none fell inside it)"
    if not inside:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no clock samples"], "samples": 0}
    return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
            "reasons": sorted({a for r in inside for a in r[4]}), "samples": len(inside),
            "power_w_max": max(r[3] for r in inside), "window": window}


class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.samples = []  # (host time, CSV line)
        self.t0 = self.t1 = None

    def start(self):
        """Start sampling every 100 ms (call before the warm-up, so that sampling runs
        by the time the timed region starts)."""
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.perf_counter(), line.strip()))

    def mark(self, t0, t1):
        """The timed region, in time.perf_counter() seconds."""
        self.t0, self.t1 = t0, t1

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        return summarize_clocks(list(self.samples), self.t0, self.t1)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return None


# ---- the oracle on the host cores ---------------------------------------------
def cpu_oracle_run(model, system, vel, steps):
    """Velocity-Verlet steps of the whole system with the FP64 oracle (one full
    force evaluation per step).  The step starts from zero forces, which changes
    the trajectory but not the work.  Returns (seconds, steps, cores)."""
    import oracle  # test infrastructure: only the baseline legs use it
    oracle.lib()
    f0 = np.zeros_like(system.pos)
    t0 = time.perf_counter()
    oracle.md(model, system, system.pos, vel, f0, steps, DT_FS)
    return time.perf_counter() - t0, steps, os.cpu_count()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    model, _, _ = workload()
    # bounded sample: a 10,000-bead box of the same water (same density, lattice
    # recipe, model and neighbour counts), one full velocity-Verlet step per timed step
    system = inputs.water_box(10_000, density=0.0334, seed=1001)
    system.masses = np.array([18.0])
    vel = inputs.maxwell_boltzmann(system, 300.0, seed=7)
    for _ in range(min(args.warmup, 1)):
        cpu_oracle_run(model, system, vel, 1)
    steps_total, secs_total = 0, 0.0
    for k in range(args.steps):
        s, st, cores = cpu_oracle_run(model, system, vel, 1)
        secs_total += s
        steps_total += st
    v = system.n * steps_total / secs_total
    sample = (f"{steps_total} FP64 velocity-Verlet steps of a {system.n}-bead box of the same water "
              f"(same density and model), one per timed step")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * secs_total / steps_total,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(workload()[1]),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---- replicas ---------------------------------------------------------------------
def replica_throughput(ms_local, units_local, dist=None, device="cpu"):
    """Whole-job throughput of independent replicas (one per rank): the units all
    ranks processed divided by the slowest rank's time.  Returns (units per second,
    job ms).  With dist (an initialised torch.distributed), every rank gets the same
    answer."""
    import torch
    ms, units = float(ms_local), float(units_local)
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        u = torch.tensor([units], dtype=torch.float64, device=device)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        ms, units = float(t.item()), float(u.item())
    return units / (ms / 1000.0), ms


# ---- our arm --------------------------------------------------------------------
def run_ours(args):
    import torch

    from paper_2603_01234_gb300 import binding

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks0 = measured_peaks()
    binding.load(build_if_missing=True)

    model, system, vel0 = workload()
    n = system.n
    m = binding.Model(model, "fp32", device=local)
    if args.tuning:  # fixed kernel variants (profiling: ncu's replay would distort the autotuner)
        tv = [int(x) for x in args.tuning.split(",")]
        binding.nep_set_tuning(m.h, 0, *tv)
    types = torch.from_numpy(system.types).to(dev)
    pos = torch.from_numpy(system.pos.copy()).to(dev)
    vel = torch.from_numpy(vel0.copy()).to(dev)
    force = torch.zeros(3, n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB

    # Every timed step starts from the same state (positions, velocities and the
    # forces at those positions), restored before the step outside the timed events
    # like the L2 flush.  The random-weight potential is not a physical water model:
    # run on, it drives the configuration away from the water structure (over 1000
    # steps the pair counts, and the force stage with them, about triple), and the
    # number would then depend on how many steps are timed.
    pos0, vel0_d = pos.clone(), vel.clone()
    force0 = None

    def restore():
        pos.copy_(pos0)
        vel.copy_(vel0_d)
        if force0 is not None:
            force.copy_(force0)

    def step(k=1, fv=1, sample=0, thermo=None):
        binding.nep_md_step(m.h, types, system.masses, system.box, system.pbc, pos, vel, force, fv, k, DT_FS,
                            sample, thermo, stream=sp)

    # pair counts of the initial configuration (for the algorithmic work)
    cnt_r, _, _ = binding.nep_neighbors(m.h, system.types, system.pos, system.box, system.pbc, 0, 1)
    cnt_a, _, _ = binding.nep_neighbors(m.h, system.types, system.pos, system.box, system.pbc, 1, 1)
    pairs_r, pairs_a = int(cnt_r.sum()), int(cnt_a.sum())

    step(k=0, fv=0)  # initial forces (the autotuner picks the kernel variants here)
    force0 = force.clone()
    tuning = binding.nep_get_tuning(m.h)
    # timed steps: each one nep_md_step call of one step, which replays the
    # handle's captured graph of the step's kernels; state restored and L2 flushed
    # before each.  The clock sampler starts before the warm-up and keeps the samples
    # of the timed region.
    clocks = Clocks(local)
    clocks.start()
    binding.nep_set_timing(m.h, 0)
    for _ in range(args.warmup):
        restore()
        flush.zero_()
        step()
    binding.nep_sync(m.h)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = time.perf_counter()
    for k in range(args.steps):
        restore()
        flush.zero_()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    binding.nep_sync(m.h)
    clocks.mark(t_start, time.perf_counter())
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    # per-stage device times: the same steps again, launched eagerly with CUDA
    # events between the stages on the launch stream (L2 flushed before each step)
    binding.nep_set_timing(m.h, 1)
    for k in range(args.steps):
        restore()
        flush.zero_()
        step()
    binding.nep_sync(m.h)
    stages, tsteps = binding.nep_get_timing(m.h)
    binding.nep_set_timing(m.h, 0)
    value, ms = replica_throughput(ms, n * args.steps, dist, dev)
    ms_step = ms / args.steps

    # steady state: 100 steps back to back through the graph-captured loop, from the
    # same state (a fixed count: a longer run drifts away from the water structure)
    steady = None
    if not args.quick:
        k2 = 100
        restore()
        step(k=k2)  # captures the chunk graph
        restore()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(k=k2)
        e1.record(stream)
        torch.cuda.synchronize()
        binding.nep_sync(m.h)
        steady = {"value": n * k2 / (e0.elapsed_time(e1) / 1000.0), "unit": UNIT, "steps": k2,
                  "how": "one nep_md_step call of k steps (CUDA graph chunks), no L2 flush"}

    # end to end through the public API with pinned host buffers (H2D + step + D2H)
    e2e = None
    if not args.quick:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
        restore()
        torch.cuda.synchronize()
        h_types, h_pos = pin(system.types), pin(pos.cpu().numpy())
        h_vel, h_force = pin(vel.cpu().numpy()), pin(force.cpu().numpy())
        thermo = pin(np.zeros((1, 12)))
        binding.nep_md_step(m.h, h_types, system.masses, system.box, system.pbc, h_pos, h_vel, h_force, 1, 1, DT_FS,
                            1, thermo)
        h_pos[:], h_vel[:], h_force[:] = pos0.cpu().numpy(), vel0_d.cpu().numpy(), force0.cpu().numpy()
        ke = 100  # from the same state, a fixed count (host buffers cannot be restored untimed)
        t0 = time.perf_counter()
        for _ in range(ke):
            binding.nep_md_step(m.h, h_types, system.masses, system.box, system.pbc, h_pos, h_vel, h_force, 1, 1,
                                DT_FS, 1, thermo)
        te = time.perf_counter() - t0
        h2d = h_types.nbytes + h_pos.nbytes + h_vel.nbytes + h_force.nbytes
        d2h = h_pos.nbytes + h_vel.nbytes + h_force.nbytes + thermo.nbytes
        e2e = {"value": n * ke / te, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "steps": ke, "how": "nep_md_step(mem=HOST, 1 step, thermo row) per step, host wall clock"}

    # the plain form: FP64 throughout, one configuration, no graph
    plain = None
    if not args.quick:
        m64 = binding.Model(model, "fp64", device=local)
        pos64, vel64 = pos0.clone(), vel0_d.clone()
        f64 = torch.zeros_like(force)
        binding.nep_md_step(m64.h, types, system.masses, system.box, system.pbc, pos64, vel64, f64, 0, 0, DT_FS,
                            0, None, stream=sp)
        binding.nep_set_timing(m64.h, 1)
        kp = 3
        binding.nep_md_step(m64.h, types, system.masses, system.box, system.pbc, pos64, vel64, f64, 1, 1, DT_FS,
                            0, None, stream=sp)
        binding.nep_sync(m64.h)
        binding.nep_set_timing(m64.h, 1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        binding.nep_md_step(m64.h, types, system.masses, system.box, system.pbc, pos64, vel64, f64, 1, kp, DT_FS,
                            0, None, stream=sp)
        b.record(stream)
        torch.cuda.synchronize()
        binding.nep_sync(m64.h)
        st64, _ = binding.nep_get_timing(m64.h)
        plain = {"value": n * kp / (a.elapsed_time(b) / 1000.0), "unit": UNIT, "steps": kp,
                 "dtype": "f64", "stages_ms_per_step": {k: v / kp for k, v in st64.items()},
                 "how": "FP64 throughout, eager launches, same workload"}
        m64.close()

    def variant_leg(params, precision, dtype, how):
        """Another model form on the same configuration, timed like the headline
        (graph replay per step, L2 flushed between steps), plus its stage times."""
        mv = binding.Model(params, precision, device=local)
        pv, vv = pos0.clone(), vel0_d.clone()
        fv_ = torch.zeros_like(force)

        def step_v(k=1, fv=1):
            binding.nep_md_step(mv.h, types, system.masses, system.box, system.pbc, pv, vv, fv_, fv, k, DT_FS,
                                0, None, stream=sp)
        step_v(k=0, fv=0)
        fv0 = fv_.clone()

        def restore_v():  # every step from the same state, as in the headline loop
            pv.copy_(pos0)
            vv.copy_(vel0_d)
            fv_.copy_(fv0)
        for _ in range(args.warmup):
            restore_v()
            flush.zero_()
            step_v()
        kv = args.steps
        evv = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(kv)]
        torch.cuda.synchronize()
        for k in range(kv):
            restore_v()
            flush.zero_()
            evv[k][0].record(stream)
            step_v()
            evv[k][1].record(stream)
        torch.cuda.synchronize()
        binding.nep_sync(mv.h)
        msv = sum(x.elapsed_time(y) for x, y in evv)
        binding.nep_set_timing(mv.h, 1)
        for k in range(kv):
            restore_v()
            flush.zero_()
            step_v()
        binding.nep_sync(mv.h)
        stv, tsv = binding.nep_get_timing(mv.h)
        binding.nep_set_timing(mv.h, 0)
        mv.close()
        return {"value": n * kv / (msv / 1000.0), "unit": UNIT, "steps": kv, "dtype": dtype,
                "stages_ms_per_step": {k: v / max(1, tsv) for k, v in stv.items()}, "how": how}

    bf16 = many_body = None
    if not args.quick:
        # BF16-weight network form
        bf16 = variant_leg(model, "bf16", "f32 + bf16 W0",
                           "BF16 hidden-layer weights, tensor-core network products; timed like the headline")
        # the same model with the four-body (l = 2) and five-body (l = 1) descriptors added
        mbp = inputs.ModelParams(**{k: getattr(model, k) for k in model.__dataclass_fields__})
        mbp.l_max_4b, mbp.l_max_5b = 2, 1
        extra = np.random.default_rng(77).standard_normal((model.n_types, model.hidden, 2 * model.n_desc_angular))
        mbp.w0 = np.concatenate([model.w0, 0.1 * extra], axis=2)
        many_body = variant_leg(mbp, "fp32", "f32",
                                f"FP32 form with four- and five-body descriptors (N_des {mbp.n_des}); "
                                "timed like the headline")

    m.close()
    configs = None
    if not args.quick and not args.no_configs and world == 1:
        sm_cfg = (peaks0 or {}).get("sm_max_mhz") or 2070.0
        configs = config_legs(dev, n_sms, sm_cfg, cpu=not args.no_cpu)
    serve = None
    if not args.quick and not args.no_serve and rank == 0:
        serve = serving_leg(local)
    if rank != 0:
        return 0

    peaks = measured_peaks()
    work = algorithmic_flops(model, pairs_r, pairs_a, n)
    dom = max(("descriptor_network", "force_virial"), key=lambda k: stages[k])
    dom_ms = stages[dom] / max(1, tsteps)
    achieved = work[dom] / (dom_ms / 1000.0) / 1e12
    sm_max = (clk.get("sm_max_mhz") or (peaks or {}).get("sm_max_mhz") or 2070.0)
    sms = n_sms
    peak = sms * 128 * 2 * sm_max * 1e6 / 1e12
    traffic = None
    import hashlib
    src = os.path.join(ROOT, "paper_2603_01234_gb300", "csrc", "evaluate.cu")
    if KERNEL_TRAFFIC["bytes_per_particle"] and dom == KERNEL_TRAFFIC["kernel"] and \
            hashlib.sha1(open(src, "rb").read()).hexdigest() == KERNEL_TRAFFIC["evaluate_cu_sha1"]:
        traffic = KERNEL_TRAFFIC["bytes_per_particle"] * n
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic, "traffic_source": KERNEL_TRAFFIC["capture"], "kernel": dom,
            "flop_per_launch": work[dom], "ms_per_launch": dom_ms, "sms": sms,
            "peak_note": FLOPS_PEAK_NOTE + f" ({sms} SMs, {sm_max:.0f} MHz max clock)"}
    if clk.get("sm_mhz"):
        roof["frac_at_median_clock"] = achieved / (sms * 128 * 2 * clk["sm_mhz"] * 1e6 / 1e12)
    # every kernel of the evaluation against its own bound, from the stage pass
    kernels = {}
    for k in ("descriptor_network", "force_virial"):
        ms_k = stages[k] / max(1, tsteps)
        kernels[k] = {"bound": "alu", "flop_per_launch": work[k], "ms_per_launch": ms_k,
                      "achieved_tflops": work[k] / (ms_k / 1000.0) / 1e12,
                      "frac": work[k] / (ms_k / 1000.0) / 1e12 / peak}
    # neighbour lists: compulsory bytes = every record read once (16 B), both lists'
    # entries written (4 B each) and the two counts (8 B) per particle
    nb_bytes = 16 * n + 4 * (pairs_r + pairs_a) + 8 * n
    ms_nb = stages["neighbor_lists"] / max(1, tsteps)
    hbm = (peaks or {}).get("hbm_gbs") or 6800.0
    kernels["neighbor_lists"] = {"bound": "hbm", "bytes_per_launch": nb_bytes, "ms_per_launch": ms_nb,
                                 "achieved_gbs": nb_bytes / (ms_nb / 1000.0) / 1e9,
                                 "peak_gbs": hbm, "frac": nb_bytes / (ms_nb / 1000.0) / 1e9 / hbm,
                                 "note": "candidate distance checks (27 cells), not bytes, bound this kernel"}

    cpu = None
    if world == 1 and not args.no_cpu:
        secs, st, cores = cpu_oracle_run(model, system, vel0, 1)
        cpu = {"value": n * st / secs, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{st} full FP64 velocity-Verlet step of all {n} beads on the host cores"}

    metric = METRIC if WORKLOAD == "water100k" and N_BEADS == 100_000 else \
        f"bead-steps/s ({WORKLOAD}, {n} particles, MD step)"
    line = {"metric": metric, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_dict(system),
            "ns_per_day": (1000.0 / ms_step) * DT_FS * 0.0864,
            # per step: kick+drift+binning, scan, scatter, in-cell ranking, neighbours,
            # descriptor+network+angular forces, radial forces+outputs+closing kick
            "gpu_launches": 7 * args.steps,
            "stages_ms_per_step": {k: v / max(1, tsteps) for k, v in stages.items()},
            "stages_how": "separate pass of the same number of steps, eager launches, CUDA events between "
                          "stages on the launch stream, L2 flushed before each step; kick_drift is the opening "
                          "kick + drift + cell binning, descriptor_network the descriptor + network + "
                          "angular-force kernel, force_virial the radial-force + output kernel (with the closing "
                          "kick), kick_sample what follows it (thermostat, thermo row; empty here)",
            "pairs_per_bead": {"radial": pairs_r / n, "angular": pairs_a / n},
            "kernel_variants": {"descriptor_blocks_per_sm": tuning[0], "force_blocks_per_sm": tuning[1],
                                "force_walk_chunk": tuning[2],
                                "chosen_by": "fixed (--tuning)" if args.tuning else "autotuner"},
            "roofline": roof, "kernels": kernels, "clocks": clk, "cpu_baseline": cpu, "e2e": e2e,
            "steady_state_graph": steady, "plain_fp64": plain, "bf16_weights": bf16, "many_body": many_body,
            "configs": configs, "serving": serve}
    print(json.dumps(line))
    return 0


# FP64 rate of the part: 1.25 TFLOP/s nominal (no measured FP64 peak exists for it)
FP64_PEAK_TFLOPS = 1.25


def md_leg(name, model, system, vel0, precision, steps, dt, dev, n_sms, sm_max, strain=None, interval=100):
    """One continuous velocity-Verlet trajectory of `steps` steps (no state restore),
    timed with CUDA events on the launch stream, in calls of `interval` steps (graph
    chunks); with strain = (axis, factor), positions and the box are rescaled by
    `factor` along `axis` after every call (nep_scale_positions on the device).
    Then a separate eager pass of 20 steps from the same start with CUDA events
    between stages, for the dominant kernel's roofline."""
    import torch

    from paper_2603_01234_gb300 import binding
    m = binding.Model(model, precision, device=dev.index or 0)
    types = torch.from_numpy(system.types).to(dev)
    pos0 = torch.from_numpy(system.pos.copy()).to(dev)
    vel0_d = torch.from_numpy(vel0.copy()).to(dev)
    pos, vel = pos0.clone(), vel0_d.clone()
    force = torch.zeros(3, system.n, dtype=torch.float64, device=dev)
    sp = torch.cuda.current_stream(dev).cuda_stream
    box = np.array(system.box, dtype=np.float64)

    def run(k, fv=1):
        binding.nep_md_step(m.h, types, system.masses, box, system.pbc, pos, vel, force, fv, k, dt, 0, None, stream=sp)

    run(0, 0)
    f0 = force.clone()
    run(min(interval, 10))  # warm-up: captures the step graph
    binding.nep_sync(m.h)
    pos.copy_(pos0)
    vel.copy_(vel0_d)
    force.copy_(f0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    done = 0
    scale = None
    if strain:
        scale = np.ones(3)
        scale[strain[0]] = strain[1]
    while done < steps:
        k = min(interval, steps - done)
        run(k)
        done += k
        if strain and done < steps:
            binding.nep_scale_positions(m.h, pos, scale, stream=sp)
            box = box * scale
    e1.record()
    torch.cuda.synchronize()
    binding.nep_sync(m.h)
    ms = e0.elapsed_time(e1)
    # stage times: a separate eager pass from the start
    box = np.array(system.box, dtype=np.float64)
    pos.copy_(pos0)
    vel.copy_(vel0_d)
    force.copy_(f0)
    binding.nep_set_timing(m.h, 1)
    run(20)
    binding.nep_sync(m.h)
    stages, tsteps = binding.nep_get_timing(m.h)
    binding.nep_set_timing(m.h, 0)
    cnt_r, _, _ = binding.nep_neighbors(m.h, system.types, system.pos, system.box, system.pbc, 0, 1)
    cnt_a, _, _ = binding.nep_neighbors(m.h, system.types, system.pos, system.box, system.pbc, 1, 1)
    tuning = binding.nep_get_tuning(m.h)
    m.close()
    n = system.n
    fp64 = precision == "fp64"
    work = algorithmic_flops(model, int(cnt_r.sum()), int(cnt_a.sum()), n, fused=not fp64)
    st = {k: v / max(1, tsteps) for k, v in stages.items()}
    dom = max(("descriptor_network", "force_virial"), key=lambda k: st[k])
    achieved = work[dom] / (st[dom] / 1000.0) / 1e12
    peak = FP64_PEAK_TFLOPS if fp64 else n_sms * 128 * 2 * sm_max * 1e6 / 1e12
    return {"workload": name, "n": n, "precision": precision, "steps": steps, "dt_fs": dt,
            "value": n * steps / (ms / 1000.0), "unit": UNIT, "ms_per_step": ms / steps,
            "ns_per_day": (1000.0 * steps / ms) * dt * 0.0864,
            "strain": None if not strain else {"axis": "xyz"[strain[0]], "factor": strain[1], "every_steps": interval},
            "pairs_per_bead": {"radial": float(cnt_r.mean()), "angular": float(cnt_a.mean())},
            "stages_ms_per_step": st, "kernel_variants": list(tuning),
            "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "peak_note": "FP64 nominal 1.25 TFLOP/s" if fp64 else
                         f"FP32 ALU: {n_sms} SMs x 128 lanes x 2 x {sm_max:.0f} MHz"},
            "how": "one continuous trajectory, calls of graph-captured step chunks, CUDA events around the run"}


def drift_leg(model, system, vel0, precision, steps, dt, dev, every=10):
    """NVE energy drift: `steps` velocity-Verlet steps from the start with a thermo
    row every `every` steps; the slope of a linear fit of E_pot + E_kin against time,
    per ns and per bead."""
    import torch

    from paper_2603_01234_gb300 import binding
    m = binding.Model(model, precision, device=dev.index or 0)
    types = torch.from_numpy(system.types).to(dev)
    pos = torch.from_numpy(system.pos.copy()).to(dev)
    vel = torch.from_numpy(vel0.copy()).to(dev)
    force = torch.zeros(3, system.n, dtype=torch.float64, device=dev)
    th = np.zeros((steps // every, 12))
    binding.nep_md_step(m.h, types, system.masses, system.box, system.pbc, pos, vel, force, 0, steps, dt, every, th,
                        stream=torch.cuda.current_stream(dev).cuda_stream)
    binding.nep_sync(m.h)
    m.close()
    t_ns = th[:, 0] * dt * 1e-6
    etot = th[:, 1] + th[:, 2]
    slope, icpt = np.polyfit(t_ns, etot, 1)
    resid = etot - (slope * t_ns + icpt)
    return {"precision": precision, "steps": steps, "dt_fs": dt, "sample_every": every,
            "drift_eV_per_ns_per_bead": slope / system.n,
            "etot_fluct_rms_eV_per_bead": float(np.sqrt(np.mean(resid ** 2))) / system.n}


def cpu_sample_leg(model, system, what):
    """The oracle (as it stands) on the host cores: one full FP64 velocity-Verlet
    step of `system`, a bounded sample of a configuration (per bead-step)."""
    vel = inputs.maxwell_boltzmann(system, 300.0, seed=7)
    secs, st, cores = cpu_oracle_run(model, system, vel, 1)
    return {"value": system.n * st / secs, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": what}


def config_legs(dev, n_sms, sm_max, cpu=True):
    """The other configurations at 1 GPU, each a continuous run: 512-bead water in
    FP64 (and FP32 beside it), the 200,000-bead four-type monolayer in FP32, with
    BF16 hidden-layer weights and (20 steps) in FP64, and the 1,000,000-particle
    nanowire over 2,000 steps with the box rescaled by 1.001 along x every 100 steps
    (and 10 steps in FP64); NVE drift over 1,000 steps of the 100,000-bead water and
    of the nanowire in FP32 and FP64.  With cpu, each configuration's
    record carries the oracle timed on a bounded sample of it (one step of the whole
    512-bead box; of an 8,000-bead monolayer and a 20,000-particle nanowire built the
    same way)."""
    out = {}
    model, system, vel = workload("water512")
    out["water512_fp64"] = md_leg("water512", model, system, vel, "fp64", 1000, 10.0, dev, n_sms, sm_max)
    out["water512_fp32"] = md_leg("water512", model, system, vel, "fp32", 1000, 10.0, dev, n_sms, sm_max)
    if cpu:
        out["water512_fp64"]["cpu_baseline"] = cpu_sample_leg(model, system, "1 full step of the 512-bead box")
    model, system, vel = workload("monolayer200k")
    out["monolayer200k_fp32"] = md_leg("monolayer200k", model, system, vel, "fp32", 500, 20.0, dev, n_sms, sm_max)
    out["monolayer200k_bf16"] = md_leg("monolayer200k", model, system, vel, "bf16", 500, 20.0, dev, n_sms, sm_max)
    out["monolayer200k_fp64"] = md_leg("monolayer200k", model, system, vel, "fp64", 20, 20.0, dev, n_sms, sm_max)
    if cpu:
        sample = inputs.monolayer(50, 40, seed=1002)
        out["monolayer200k_fp32"]["cpu_baseline"] = cpu_sample_leg(
            model, sample, f"1 full step of a {sample.n}-bead monolayer built like the 200,000-bead one")
    model, system, vel = workload("nanowire1M")
    out["nanowire1M_fp32_strain"] = md_leg("nanowire1M", model, system, vel, "fp32", 2000, 5.0, dev, n_sms, sm_max,
                                           strain=(0, 1.001), interval=100)
    out["nanowire1M_fp64"] = md_leg("nanowire1M", model, system, vel, "fp64", 10, 5.0, dev, n_sms, sm_max)
    if cpu:
        sample = inputs.nanowire(20_000, seed=1003)
        out["nanowire1M_fp32_strain"]["cpu_baseline"] = cpu_sample_leg(
            model, sample, f"1 full step of a {sample.n}-particle nanowire built like the 1,000,000-particle one")
    out["drift"] = {"nanowire1M": [drift_leg(model, system, vel, "fp32", 1000, 5.0, dev),
                                   drift_leg(model, system, vel, "fp64", 1000, 5.0, dev)]}
    model, system, vel = workload("water100k")
    out["drift"]["water100k"] = [drift_leg(model, system, vel, "fp32", 1000, 10.0, dev),
                                 drift_leg(model, system, vel, "fp64", 1000, 10.0, dev)]
    return out


def serving_leg(device, n_requests=4096, fractions=(0.25, 0.5, 0.75, 0.9), repeats=5, lanes=2):
    """Served stream: n_requests energy/force/virial requests, bead counts
    log-uniform in [64, 4096], half water-like cubes (model 0), half four-type
    monolayer patches (model 1); host buffers in and out (each lane packs its batches
    into page-locked buffers).  Saturation throughput (all requests queued at t = 0)
    and p50/p99 latency under Poisson arrivals at fractions of each form's own
    saturation rate, each load repeated `repeats` times with fresh arrival times
    (median and range reported), for the batched server (`lanes` lanes, admission by
    the library's workspace bytes), for the same server with the requests'
    configurations and results on the GPU (device_resident: no host copies), and for
    one launch sequence per request."""
    import torch

    from paper_2603_01234_gb300 import serving

    m_water = inputs.random_model(n_types=1, hidden=30, rc_radial=8.0, rc_angular=5.0, seed=1)
    m_mono = inputs.random_model(n_types=4, hidden=50, rc_radial=15.0, rc_angular=11.0, seed=2)
    stream = inputs.request_stream(n_requests=n_requests, seed=1004)
    dev = torch.device("cuda", device)
    stream_dev = [(mi, inputs.System(pos=torch.from_numpy(np.ascontiguousarray(s.pos)).to(dev),
                                     types=torch.from_numpy(s.types.astype(np.int32)).to(dev), box=s.box,
                                     pbc=s.pbc)) for mi, s in stream]
    out = {"requests": n_requests, "particles": int(sum(s.n for _, s in stream)), "repeats_per_load": repeats,
           "workload": "log-uniform 64-4096 beads; water cubes (1 type, H=30, r_c 8/5) and 4-type monolayer "
                       "patches (H=50, r_c 15/11), 50/50; host buffers (device_resident: CUDA tensors)"}
    forms = {"batched": dict(lanes=lanes, lane_bytes=2 << 30, max_requests=4096),
             "batched_device_resident": dict(lanes=lanes, lane_bytes=2 << 30, max_requests=4096,
                                             device_resident=True),
             "one_launch_per_request": dict(lanes=1, lane_bytes=2 << 30, max_requests=1)}
    streams = {name: (stream_dev if kw.get("device_resident") else stream) for name, kw in forms.items()}
    sat = {}
    for name, kw in forms.items():
        srv = serving.Server([m_water, m_mono], "fp32", device=device, keep_results=False, **kw)
        stream = streams[name]
        # warm-up: the whole stream once, so every lane's workspace and staging are
        # sized (steady-state serving) before the timed runs
        warm = [serving.Request(k, mi, s) for k, (mi, s) in enumerate(stream)]
        srv.serve(warm, np.zeros(len(warm)))
        reqs = [serving.Request(k, mi, s) for k, (mi, s) in enumerate(stream)]
        st = srv.serve(reqs, np.zeros(len(reqs)))
        sat[name] = st
        out[name] = {"lanes": kw["lanes"],
                     "saturation": {"particles_per_s": st.throughput, "requests_per_s": st.n_requests / st.wall_s,
                                    "batches": st.batches, "mean_requests_per_batch": st.mean_batch_requests,
                                    "p50_ms": 1e3 * st.pct(50), "p99_ms": 1e3 * st.pct(99)},
                     "poisson": []}
        srv.close()
    for name, kw in forms.items():
        srv = serving.Server([m_water, m_mono], "fp32", device=device, keep_results=False, **kw)
        stream = streams[name]
        warm = [serving.Request(k, mi, s) for k, (mi, s) in enumerate(stream)]
        srv.serve(warm, np.zeros(len(warm)))
        rate_sat = sat[name].n_requests / sat[name].wall_s  # each form at fractions of its own saturation
        for f in fractions:
            rate = f * rate_sat
            p50, p99, thr, mb = [], [], [], []
            for rep in range(repeats):
                reqs = [serving.Request(k, mi, s) for k, (mi, s) in enumerate(stream)]
                st = srv.serve(reqs, serving.poisson_arrivals(len(reqs), rate, seed=7 + 1000 * rep))
                p50.append(1e3 * st.pct(50))
                p99.append(1e3 * st.pct(99))
                thr.append(st.throughput)
                mb.append(st.mean_batch_requests)
            out[name]["poisson"].append({
                "rate_req_per_s": rate, "fraction_of_own_saturation": f,
                "p50_ms": statistics.median(p50), "p50_ms_range": [min(p50), max(p50)],
                "p99_ms": statistics.median(p99), "p99_ms_range": [min(p99), max(p99)],
                "particles_per_s": statistics.median(thr), "mean_requests_per_batch": statistics.median(mb)})
        srv.close()
    return out


def run_drift(args, n_steps=1000, every=10):
    """NVE energy drift of the workload in the FP32 and FP64 forms: n_steps
    velocity-Verlet steps from 300 K, thermo row every `every` steps; the drift is
    the slope of a linear fit of E_pot + E_kin against time, per ns and per bead."""
    import torch

    from paper_2603_01234_gb300 import binding
    binding.load(build_if_missing=True)
    dev = torch.device("cuda", 0)
    model, system, vel0 = workload()
    out = {"metric": "NVE energy drift", "workload": WORKLOAD, "n": system.n, "dt_fs": DT_FS, "steps": n_steps,
           "forms": {}}
    for precision in ("fp32", "fp64"):
        m = binding.Model(model, precision)
        types = torch.from_numpy(system.types).to(dev)
        pos = torch.from_numpy(system.pos.copy()).to(dev)
        vel = torch.from_numpy(vel0.copy()).to(dev)
        force = torch.zeros(3, system.n, dtype=torch.float64, device=dev)
        th = np.zeros((n_steps // every, 12))
        st = torch.cuda.current_stream(dev).cuda_stream
        t0 = time.perf_counter()
        binding.nep_md_step(m.h, types, system.masses, system.box, system.pbc, pos, vel, force, 0, n_steps, DT_FS,
                            every, th, stream=st)
        binding.nep_sync(m.h)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        t_ns = th[:, 0] * DT_FS * 1e-6
        etot = th[:, 1] + th[:, 2]
        slope, icpt = np.polyfit(t_ns, etot, 1)
        resid = etot - (slope * t_ns + icpt)
        temp = 2.0 * th[:, 2] / ((3 * system.n - 3) * inputs.KB_EV)
        out["forms"][precision] = {
            "drift_eV_per_ns_per_bead": slope / system.n, "etot_first": etot[0], "etot_last": etot[-1],
            "etot_fluct_rms_eV_per_bead": float(np.sqrt(np.mean(resid ** 2))) / system.n,
            "epot_change_eV_per_bead": (th[-1, 1] - th[0, 1]) / system.n,
            "temperature_first_K": temp[0], "temperature_last_K": temp[-1],
            "bead_steps_per_s_wall": system.n * n_steps / wall}
        m.close()
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true", help="skip the steady-state, e2e and FP64 legs")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-serve", action="store_true", help="skip the served-stream leg")
    ap.add_argument("--no-configs", action="store_true", help="skip the other configurations' runs")
    ap.add_argument("--workload", default="water100k", choices=sorted(WORKLOADS),
                    help="the metric is quoted on water100k; the others are further configurations")
    ap.add_argument("--drift", action="store_true", help="NVE energy-drift run (1000 steps, FP32 and FP64)")
    ap.add_argument("--tuning", default=None, help="fix the kernel variants 'D,F[,C]' (resident blocks per SM of "
                                                    "the descriptor and radial-force kernels, and the radial "
                                                    "kernel's walk chunk 4 or 8); default: autotuned")
    ap.add_argument("--n-beads", type=int, default=N_BEADS,
                    help="size of the water box (profiling captures only; the metric is quoted at 100000)")
    args = ap.parse_args()
    globals()["N_BEADS"] = args.n_beads
    globals()["WORKLOAD"] = args.workload
    globals()["DT_FS"] = WORKLOADS[args.workload][1]
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.drift:
        return run_drift(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
