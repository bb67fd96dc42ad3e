"""The multi-GPU form of the benchmark is replicas only (each rank parses its
own copy of the workload, no data exchange): the ranks agree on the step time
(the slowest rank's) and report the throughput of all replicas together.
Checked here with two gloo ranks on the CPU."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    import bench

    w, r, _ = bench.dist_setup("gloo")
    try:
        step_ms, kern_ms = bench.max_over_ranks([10.0 + 5 * r, 8.0 - r], w, "cpu")
        q.put((r, w, step_ms, kern_ms, bench.whole_job_rate(w, 1_000_000_000, step_ms)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, step_ms, kern_ms, rate in got:
        assert w == world
        assert step_ms == 15.0 and kern_ms == 8.0  # each timing's maximum over the ranks
        assert rate == pytest.approx(2 * 1e9 / 15e-3 / 1e9)  # both replicas' bytes in the slowest time


def test_single_process_is_unchanged():
    import bench

    assert bench.max_over_ranks([3.0, 4.0], 1, "cpu") == [3.0, 4.0]
    assert bench.whole_job_rate(1, 2_000_000_000, 1000.0) == pytest.approx(2.0)
