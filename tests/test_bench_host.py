"""Host logic of bench.py: the N > 1 aggregation over replicas, on CPU with gloo."""

import json
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (r + 1) seconds for 1e6 points
        v, slowest = bench.whole_job_throughput(rank + 1.0, 1_000_000, dist, "cpu")
        out[rank] = (v, slowest)
    finally:
        dist.destroy_process_group()


def test_whole_job_throughput_single_process():
    v, s = bench.whole_job_throughput(2.0, 4_000_000)
    assert s == 2.0 and v == pytest.approx(2.0)


def test_whole_job_throughput_two_gloo_ranks_takes_the_slowest_rank():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    # both ranks see the slowest rank's 2 s; the job processed 2 x 1e6 points
    for r in range(world):
        v, slowest = res[r]
        assert slowest == 2.0
        assert v == pytest.approx(world * 1e6 / 2.0 / 1e6)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), {"workload": "c1", "warmup": 3, "steps": 1, "gpus": 2})()
    assert bench.run_reference(args) == 0


def test_reference_arm_prints_one_line_with_the_contract_keys(monkeypatch, capsys):
    # rank 0 times the oracle on a bounded sample of the workload (C1, N = 256, here) and
    # prints the same line as the main arm, with impl = reference and its own e2e
    monkeypatch.setenv("RANK", "0")
    args = type("A", (), {"workload": "c1", "warmup": 3, "steps": 1, "gpus": 1})()
    assert bench.run_reference(args) == 0
    out = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(out) == 1
    line = json.loads(out[0])
    assert line["impl"] == "reference" and line["metric"] == "FMM matvec Mpts/s" and line["unit"] == "Mpts/s"
    assert line["value"] > 0 and line["higher_is_better"] is True and line["steps"] == 1
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
