"""The multi-GPU bookkeeping of bench.py on CPU (gloo, world size 2).

A product of the workload's size is one GPU's work and the library has no
exchange step, so N GPUs run N independent replicas: the job's time is the
slowest rank's and its throughput counts every rank's product.  These tests
run that bookkeeping with the gloo backend on two CPU processes; the product
itself needs a GPU and is covered by the -m gpu tests.
"""
import importlib.util
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    ms_total = [240.0, 260.0][rank]          # the second rank is slower
    m = b.max_over_ranks(ms_total, world, "cpu")
    value = b.job_value(world, m / 10)
    dist.barrier()
    if rank == 0:
        with open(out_path, "w") as f:
            json.dump({"max": m, "value": value}, f)
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_count_every_product(tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "r.json")
    mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    r = json.load(open(out))
    b = _bench()
    assert r["max"] == 260.0
    n2k = b.N * b.N * b.K
    assert abs(r["value"] - 2 * n2k / 26.0e-3 / 1e9) < 1e-6 * r["value"]


def test_single_rank_needs_no_process_group():
    b = _bench()
    assert b.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert b.job_value(1, 25.0) == b.N * b.N * b.K / 25.0e-3 / 1e9


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun the reference arm (the CPU oracle) runs on rank 0
    alone; the other ranks exit 0 at once, printing nothing."""
    b = _bench()
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), {"steps": 1, "warmup": 0, "gpus": 2})()
    assert b.run_reference(args) == 0
    assert capsys.readouterr().out == ""
