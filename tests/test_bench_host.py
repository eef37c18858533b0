"""Host-side logic of bench.py's multi-process (replica) path, on CPU with the
gloo backend and two ranks: the job time is the slowest rank's, the rate
counts every rank's particles, and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [10.0 + rank, 20.0 - 5.0 * rank]            # rank 0: (10, 20), rank 1: (11, 15)
    got = bench.max_over_ranks(local, world, torch, dist, "cpu")
    out[rank] = got
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_gloo_two_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == [11.0, 20.0]
    import bench
    # 2 ranks x 1000 particles x 5 steps in 11 ms
    assert bench.job_rate(2, 1000, 5, 11.0) == pytest.approx(2 * 1000 * 5 / 0.011)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    class A:
        particles = 1000
        steps = 1
        warmup = 0
        workload = "gas-cloud"
    bench.run_reference(A())                       # returns at once: no work, no output
    assert capsys.readouterr().out == ""


def test_fit_traffic_only_where_it_was_captured():
    """The ncu traffic figure describes the split FP32 pass with the plain
    estimator on the gas cloud; every other configuration reports none."""
    import bench
    n = 2_000_000
    assert bench.fit_traffic("fp32", "plain", True, "gas-cloud", n) == bench.FIT_TRAFFIC_BPP * n
    assert bench.fit_traffic("fp32", "plain", False, "gas-cloud", n) is None
    assert bench.fit_traffic("fp64", "plain", True, "gas-cloud", n) is None
    assert bench.fit_traffic("fp32", "mlp", True, "gas-cloud", n) is None
    assert bench.fit_traffic("fp32", "plain", True, "jet-snapshot", n) is None
