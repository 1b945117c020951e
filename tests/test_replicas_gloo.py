"""Multi-GPU runs are independent replicas (no data-path collective): the bench's
whole-job throughput is the units of all ranks over the slowest rank's time.  The
aggregation runs here as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = 10.0 + 5.0 * rank          # rank 1 is the slower one
    units_local = 1000 * (100 + rank)    # bead-steps of this rank's replica
    value, ms = bench.replica_throughput(ms_local, units_local, dist)
    dist.barrier()
    out[rank] = (value, ms)
    dist.destroy_process_group()


def test_two_replicas_aggregate_over_gloo():
    world, port = 2, free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    want_ms = 15.0
    want_value = (1000 * 100 + 1000 * 101) / (want_ms / 1000.0)
    for r in range(world):
        value, ms = out[r]
        assert ms == want_ms
        assert value == pytest.approx(want_value, rel=1e-12)


def test_single_replica_is_plain_throughput():
    import bench
    value, ms = bench.replica_throughput(20.0, 5000)
    assert ms == 20.0 and value == pytest.approx(5000 / 0.020)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun only rank 0 times the oracle and prints; other ranks exit 0."""
    import argparse

    import bench
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(steps=1, warmup=0, gpus=2)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
