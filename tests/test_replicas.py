"""The N > 1 path of bench.py without a GPU: world_size-2 gloo ranks on the
CPU, rendezvous on 127.0.0.1.  The grid step does not shard in this build
(one GPU per run): N ranks are independent replicas, so the only exchanges
are the timing barrier and the max over ranks of the timed region; the job's
value is N x the units of one replica over that max.  The reference arm runs
on rank 0 alone; the other ranks exit at once without work."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench._dist = dist
    bench.barrier()
    seconds = 1.0 + rank                      # rank 1 is the slow replica
    slowest = bench.max_over_ranks(torch, seconds)
    value = bench.job_value(world, 1e6 * 50, slowest)
    out[rank] = (slowest, value)
    bench.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_agree_on_the_slowest_time():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:      # no fork of this multi-threaded process
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1]
    slowest, value = res[0]
    assert slowest == 2.0
    assert value == pytest.approx(2 * 50.0 / 2.0)   # 2 replicas x 50 M units in 2 s


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    called = []
    monkeypatch.setattr(bench, "cpu_baseline", lambda *a, **k: called.append(1))
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), {"steps": 2, "warmup": 3, "gpus": 2})()
    assert bench.run_reference(args) == 0
    assert not called
