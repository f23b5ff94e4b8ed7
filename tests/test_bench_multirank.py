"""bench.py's multi-rank host logic on CPU (gloo, world size 2): replicas, slowest-rank time,
whole-job throughput; the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [10.0, 12.5][rank]  # rank 1 is the slower replica
    max_ms, value = bench.replica_throughput(ms, nodes=1000, steps=20, dist=dist, device="cpu")
    out[rank] = (max_ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_takes_the_slowest_rank_and_all_nodes():
    mp_ctx = mp.get_context("spawn")
    manager = mp_ctx.Manager()
    out = manager.dict()
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        max_ms, value = out[r]
        assert max_ms == 12.5
        assert value == pytest.approx(1000 * 20 * world / 0.0125)


def test_replica_throughput_single_process():
    import bench
    assert bench.replica_throughput(5.0, nodes=10, steps=4) == (5.0, 10 * 4 / 0.005)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import bench
    ns = type("A", (), {"workload": "tgv_32c_p4", "warmup": 0, "steps": 1})()
    bench.run_reference(ns, rank=1, world=2)  # other ranks exit without work or output
    assert capsys.readouterr().out == ""
