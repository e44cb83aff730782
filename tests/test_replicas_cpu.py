"""Replicas across ranks (the multi-GPU mode of the benchmark; the walk needs
no data exchange): two gloo ranks on CPU check the max-over-ranks timing and
the whole-job rate, and that only rank 0 of the reference arm does work."""
import json
import os
import socket
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_replicas_report_the_slowest_rank():
    torch = pytest.importorskip("torch")
    import multiprocessing as mp

    import replica_workers
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=replica_workers.replica_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, env, ms, rate in out:
        assert env == (2, rank, rank)
        assert ms == 1.5                      # the slower rank's time
        assert rate == 2 * 1000.0 / 1.5e-3    # units of both ranks over that time


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1, None) == 3.25
    assert bench.job_rate(10.0, 1, 2.0) == 5000.0


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench
    args = types.SimpleNamespace(ref_targets=4, warmup=1, steps=1, theta=0.5, workload="uniform4096")
    assert bench.run_reference(args, None, 2, 1) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_line(capsys):
    sys.path.insert(0, ROOT)
    import bench
    import ics
    w = ics.make("uniform4096", 500)
    args = types.SimpleNamespace(ref_targets=50, warmup=1, steps=2, theta=0.5, workload="uniform4096")
    assert bench.run_reference(args, w, 1, 0) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
