"""bench.py's multi-rank bookkeeping on CPU: two gloo ranks (one process
each, as torchrun would start them) agree on the slowest rank's time, the
whole-job rate counts every rank's units, and the reference arm runs on rank
0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w, r, loc = bench.dist_env()
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, w, "cpu")
        rate = bench.whole_job_rate(1000, 4, w, ms)
        q.put((r, loc, w, ms, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[0] for g in got] == [0, 1] and [g[1] for g in got] == [0, 1]
    for r, loc, w, ms, rate in got:
        assert w == 2 and ms == 15.0
        # 1000 units x 4 steps on each of 2 ranks in 15 ms
        assert rate == pytest.approx(8000 / 0.015)


def test_reference_arm_is_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        gpus, steps, warmup = 2, 1, 0
    bench.bench_reference(A())
    assert capsys.readouterr().out == ""


def test_reference_arm_prints_the_contract_line():
    # rank 0, N = 1: one JSON line timing the FP64 oracle on a bounded sample,
    # on the same workload, metric and unit as the CUDA arm
    import json
    import subprocess
    sys.path.insert(0, ROOT)
    import bench
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=300, check=True).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 1 and line["steps"] == 1
    assert line["metric"] == bench.METRIC and line["unit"] == "events/s"
    assert line["config"]["workload"] == bench.WORKLOADS[bench.HEADLINE][0]
    assert line["higher_is_better"] is True and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "events/s",
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
