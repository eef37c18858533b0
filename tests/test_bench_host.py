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
    """An ncu traffic figure describes the split FP32 pass with the plain
    estimator on the gas cloud; every other configuration, and a kernel whose
    figure is stale (None), reports none."""
    import bench
    n = 2_000_000
    assert bench.fit_traffic("fp32", "plain", True, "gas-cloud", n, 900.0) == 900.0 * n
    assert bench.fit_traffic("fp32", "plain", True, "gas-cloud", n, None) is None
    assert bench.fit_traffic("fp32", "plain", False, "gas-cloud", n, 900.0) is None
    assert bench.fit_traffic("fp64", "plain", True, "gas-cloud", n, 900.0) is None
    assert bench.fit_traffic("fp32", "mlp", True, "gas-cloud", n, 900.0) is None
    assert bench.fit_traffic("fp32", "plain", True, "jet-snapshot", n, 900.0) is None


def test_fit_flop_model_counts_the_work_the_kernels_do():
    """The flop model charges the normal equations per neighbour row, the
    correction pass only on the refined share, and the one-sided fits only on
    the plain-estimator share; each part by its operation count."""
    import bench
    m = 44.7
    full = bench.fit_flops_per_particle(m, 1.0, 1.0)
    none = bench.fit_flops_per_particle(m, 0.0, 0.0)
    # per row of the central fit: 36 to build it, 180 for the 90 FMA of the Gram
    # matrix and A^T B; factor 285 and solve 774 once
    assert none == m * 216 + 285 + 774 + 500
    # the correction pass: the row again (36) and 2 x 45 FMA, and a solve
    assert bench.fit_flops_per_particle(m, 1.0, 0.0) - none == m * (36 + 180) + 774
    # one-sided: 6 fits of 8 rows, 138 flops a row, and 30 for each back substitution
    assert bench.fit_flops_per_particle(m, 0.0, 1.0) - none == 6 * (8 * 138 + 30)
    assert 17_000 < bench.fit_flops_per_particle(m, 0.03, 1.0) < 20_000 < full


def test_workload_settings():
    """Each workload's configuration: the gas cloud keeps the nearest k_max = 64
    neighbours; the jet workloads, whose configuration quotes 20-80
    neighbours, take k_max = 80 with the octant-balanced selection unless
    --select says otherwise; the estimator comparison is its own mode."""
    import bench
    a = bench.parse([])
    bench.select_workload(a)
    assert (bench.K_MAX, bench.SELECT, a.particles) == (64, "nearest", 2_000_000)
    assert a.compare_estimators == 0
    for w in ("jet-snapshot", "jet-inflow"):
        a = bench.parse(["--workload", w])
        bench.select_workload(a)
        assert (bench.K_MAX, bench.SELECT, a.particles) == (80, "octant", 8_000_000)
        cfg = bench.config_dict(a.particles)
        assert cfg["k_max"] == 80 and cfg["select"] == "octant"
    a = bench.parse(["--workload", "jet-snapshot", "--select", "nearest"])
    bench.select_workload(a)
    assert bench.SELECT == "nearest"
    a = bench.parse(["--compare-estimators", "200", "--particles", "400000"])
    bench.select_workload(a)
    assert (a.compare_estimators, a.particles, bench.K_MAX) == (200, 400_000, 64)
    bench.select_workload(bench.parse([]))          # back to the default workload for later tests
