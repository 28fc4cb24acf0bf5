"""Host logic of the multi-GPU bench (replicas, no data-path collective),
run as two gloo ranks on the CPU: each rank solves its own batch, the job
time is the slowest rank's and the value counts the RHS of all ranks."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = 100.0 + 50.0 * rank          # rank 1 is the slowest
        ms_all, value = bench.aggregate(ms_local, world, 64, dist, "cpu")
        out[rank] = (ms_all, value, bench.source_seed(rank))
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        ms_all, value, seed = out[rank]
        assert ms_all == 150.0                      # MAX over ranks
        assert abs(value - world * 64 / 0.150) < 1e-9
    assert out[0][2] == 1 and out[1][2] != out[0][2]   # independent batches, rank 0 = headline


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "oracle_sample", lambda *a, **k: called.append(1))
    class A:
        n, nrhs, warmup, steps, gpus = 31, 2, 1, 1, 2
    bench.run_reference(A())
    assert not called
