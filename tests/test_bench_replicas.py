"""The multi-GPU path of bench.py (independent replicas, one per rank) on the
CPU: two gloo ranks with different local times agree on the whole-job rate
(the units of every rank over the slowest rank's time, max over ranks), and
the reference arm does its work on rank 0 only."""
import argparse
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica(rank, world, port, local_ms, units, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    rate, slowest = bench.whole_job_rate(local_ms, units, world, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, rate, slowest))


def test_two_replicas_report_the_slowest_rank():
    world, units = 2, 1000
    local = [10.0, 15.0]
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_replica, args=(r, world, port, local[r], units, q)) for r in range(world)]
    for p in ps:
        p.start()
    got = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, slowest in got:
        assert slowest == max(local)
        assert rate == pytest.approx(world * units / (max(local) * 1e-3))


def test_single_rank_rate():
    import bench
    rate, slowest = bench.whole_job_rate(12.0, 600, 1, "cpu")
    assert slowest == 12.0
    assert rate == pytest.approx(600 / 12e-3)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    """A rank other than 0 exits 0 at once, without starting the oracle."""
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = argparse.Namespace(gpus=2, steps=1, warmup=0, batch_count=256, impl="reference")
    assert bench.run_reference(args) == 0
