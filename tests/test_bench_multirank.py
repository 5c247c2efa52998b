"""The benchmark's multi-rank path on the CPU (gloo, world size 2): replicas
synchronise with a barrier, the step time is the slowest rank's, the job
value counts all ranks' work, and the reference arm runs on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    r, w, local = bench._dist()
    assert (r, w, local) == (rank, world, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    barrier, max_over_ranks = bench._collectives(world, torch.device("cpu"))
    barrier()
    ms = max_over_ranks(10.0 + 5.0 * rank)          # the slowest rank decides
    value = bench.job_value(world, 1000.0, ms)
    # the reference arm: rank 0 alone runs and prints; the others return at once
    class A:
        steps, warmup, ref_instances = 1, 0, 2
    buf = io.StringIO()
    if rank != 0:
        with redirect_stdout(buf):
            bench.run_reference(A, rank, world)
    barrier()
    dist.destroy_process_group()
    out.put((rank, ms, value, buf.getvalue()))


def test_two_replicas_max_time_and_job_value():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value, printed in res:
        assert ms == 15.0                            # max over ranks, seen by both
        assert value == pytest.approx(2 * 1000.0 / 0.015)
        if rank != 0:
            assert printed == ""                     # reference arm silent off rank 0


def test_single_rank_collectives_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    barrier, max_over_ranks = bench._collectives(1, torch.device("cpu"))
    barrier()
    assert max_over_ranks(3.5) == 3.5
    assert bench.job_value(1, 100.0, 50.0) == pytest.approx(2000.0)


def test_reference_arm_line_on_rank_zero():
    """Rank 0 of the reference arm prints one JSON line with the contract's
    keys: the oracle timed on the host cores, its own cpu_baseline, and an
    e2e figure with no host-device traffic."""
    import json
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup, ref_instances = 2, 0, 2
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(A, 0, 1)
    lines = [l for l in buf.getvalue().splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    # the same workload description as the GPU arm's line
    assert d["config"] == bench._ntt_config("replicas x1")
    assert "2 of 1024 instances" in d["cpu_baseline"]["sample"]
