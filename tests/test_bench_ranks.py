"""The N-GPU bench path runs independent replicas (the step has no exchange on
one GPU; see the multi-GPU note of the design): whole-job throughput is every
rank's updates over the slowest rank's time.  Checked with two gloo ranks on
the CPU."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        ms = [120.0, 150.0][rank]  # rank 1 is the slowest
        out[rank] = b.replica_throughput(ms, 1000, 200, world, torch.device("cpu"))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_replicas_take_the_slowest_rank():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    for r in (0, 1):
        ms_max, mlups = out[r]
        assert ms_max == 150.0
        assert mlups == pytest.approx(1000 * 200 * 2 / 0.150 / 1e6)


def test_single_replica():
    b = _bench()
    ms_max, mlups = b.replica_throughput(100.0, 5000, 10, 1, torch.device("cpu"))
    assert ms_max == 100.0 and mlups == pytest.approx(5000 * 10 / 0.1 / 1e6)
