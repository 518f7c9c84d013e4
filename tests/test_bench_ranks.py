"""The bench's multi-rank bookkeeping (replicas: max time over ranks, total
work summed) with two gloo ranks on the CPU, and the reference arm's rank
rule (only rank 0 works)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


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
    import bench
    t, w = bench.reduce_over_ranks(5.0 + 10.0 * rank, 100 * (rank + 1), "cpu")
    out[rank] = (t, w)
    dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    assert out[0] == (15.0, 300.0) and out[1] == (15.0, 300.0)


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_over_ranks(7.0, 42) == (7.0, 42.0)


def test_reference_arm_other_ranks_do_nothing():
    import argparse

    import bench
    args = argparse.Namespace(workload="single_n2000_d3", steps=1, warmup=0, gpus=2)
    assert bench.run_reference(args, rank=1, world=2) == 0


def test_reference_arm_line_on_the_small_workload(capsys):
    # the oracle timed on the host cores: one JSON line with the contract's keys
    import argparse
    import json

    import bench
    args = argparse.Namespace(workload="single_n2000_d3", steps=1, warmup=1, gpus=1)
    assert bench.run_reference(args, rank=0, world=1) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["n_gpus"] == 1
    for key in ("metric", "unit", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"] == "single_n2000_d3"
