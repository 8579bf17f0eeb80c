"""Host logic of bench.py's multi-GPU mode (independent replicas, no data-path
collective): the timed region is the slowest rank's, the value counts every
rank's columns, and the reference arm runs on rank 0 only.  Two gloo ranks on
the CPU stand in for two GPUs."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_seconds = [3.0, 5.0][rank]  # rank 1 is the slower replica
        slowest = bench.max_over_ranks(local_seconds, dist, "cpu")
        q.put((rank, slowest, bench.whole_job_rate(world, 12, 4, slowest)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    # both ranks see the slower replica's 5 s; the job solved 2 x 12 x 4 columns
    assert [g[1] for g in got] == [5.0, 5.0]
    assert got[0][2] == pytest.approx(2 * 12 * 4 / 5.0)


def test_without_a_group_the_local_time_stands():
    assert bench.max_over_ranks(2.5) == 2.5
    assert bench.whole_job_rate(1, 12, 5, 10.0) == pytest.approx(6.0)


def test_reference_arm_prints_on_rank_zero_only(capsys):
    class A:
        workload, steps, warmup = "wilson_8c16_L12", 1, 0

    bench.run_reference(A(), dict(bench.WORKLOADS["wilson_8c16_L12"]), rank=1, world=2)
    assert capsys.readouterr().out == ""


def test_reference_line_keeps_the_contract(capsys, monkeypatch):
    """The reference arm (the oracle on the host cores) prints one JSON line
    with the contract's keys; a one-iteration sample of the 8^3 x 16 workload
    keeps the test short."""
    import json

    real = bench.oracle_sample
    monkeypatch.setattr(bench, "oracle_sample", lambda cfg, iters: real(cfg, iters, n_iter=1))

    class A:
        workload, steps, warmup = "wilson_8c16_L12", 1, 0

    bench.run_reference(A(), dict(bench.WORKLOADS["wilson_8c16_L12"]), rank=0, world=1)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == bench.UNIT
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["config"]["workload"] == "wilson_8c16_L12"
