"""The multi-replica bench path on CPU: world_size-2 gloo process group.

bench.py runs one independent replica per rank (the factorization does not
shard); the job's time is the slowest rank's and its throughput counts every
rank's steps.  The reference arm does its work on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 10.0 * (rank + 1)          # rank 1 is the slow one
    m = bench.max_over_ranks(local_ms, dist, "cpu")
    q.put((rank, m, bench.job_rate(5, world, m)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [r for r, _, _ in out] == [0, 1]
    for _, m, v in out:
        assert m == 20.0                   # both ranks see the slowest time
        assert v == pytest.approx(2 * 5 / 0.020)


def test_single_process_and_reference_arm_rank_gate(monkeypatch):
    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5
    assert bench.job_rate(10, 1, 100.0) == pytest.approx(100.0)
    monkeypatch.setenv("RANK", "1")
    # a non-zero rank of the reference arm returns at once, without work
    assert bench.run_reference(type("A", (), {})()) == 0


def test_parallel_oracle_baseline_counts_every_set():
    # the batched workload's CPU baseline: value sets spread over processes
    cpu = bench.cpu_batched_baseline("grid32_natural", list(range(5)), sigma=0.0, base_seed=None, cores=2)
    assert cpu["cores"] == 2 and cpu["kind"] == "oracle" and cpu["value"] > 0
    assert cpu["sample"].startswith("5 value sets")
    one = bench.cpu_batched_baseline("grid32_natural", [3], sigma=0.0, base_seed=None, cores=8)
    assert one["cores"] == 1                  # never more processes than sets
