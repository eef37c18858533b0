"""Fit schedules and the autotuner.

The split schedule (central kernel + compacted plain-stage kernel) executes the
same per-particle arithmetic as the fused kernel, so both must give the same
state bit for bit, with the plain estimator (every particle takes the plain
stage) and with the learned estimator (particles the gate clears are finished
by the first kernel).  The autotuner must leave the particle state and the
counters as they were.
"""
import numpy as np
import pytest

from paper_2206_11998_gb300 import inputs, lp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from tests.gpu_util import ensure_built
    ensure_built()


N = 60_000


def _cloud():
    return inputs.gas_cloud_3d(N, seed=21)


def _cfg(st, **kw):
    return lp.make_config(3, N, kappa=2.2, k_max=64, gamma=5.0 / 3.0, s_ref=inputs.field_scales(st), **kw)


def _run(st, sched, steps=2, params=None, **kw):
    ctx = lp.Context(_cfg(st, **kw))
    if params is not None:
        ctx.mlp_set_params(params)
    ctx.set_schedule(sched)
    assert ctx.schedule() == sched
    ps = lp.ParticleSet.from_state(st)
    flag = torch.empty(N, dtype=torch.uint8, device="cuda")
    phi = torch.empty((N, 5), dtype=torch.float32, device="cuda")
    for _ in range(steps):
        ctx.step(ps, dt=0.0, cfl=0.4, flag=flag, phi=phi)
    torch.cuda.synchronize()
    out = (ps.to_state(N), flag.cpu().numpy(), phi.cpu().numpy(), ctx.stats())
    ctx.close()
    return out


def _same(a, b):
    (ga, fa, pa, sa), (gb, fb, pb, sb) = a, b
    assert np.array_equal(ga["id"], gb["id"])
    for f in ("V", "P", "m"):
        assert np.array_equal(ga[f], gb[f]), f
    for d in range(3):
        assert np.array_equal(ga["x"][d], gb["x"][d]), d
        assert np.array_equal(ga["u"][d], gb["u"][d]), d
    assert np.array_equal(fa, fb)
    assert np.array_equal(pa, pb)
    for k in ("n_flagged", "n_fp64_redo", "n_nonfinite", "n_mlp_skip", "n_mlp_uncertain", "n_mlp_miss", "steps"):
        assert sa[k] == sb[k], k


@pytest.mark.parametrize("prec", [lp.PREC_FP32, lp.PREC_FP64])
def test_split_equals_fused_plain_estimator(prec):
    st = _cloud()
    a = _run(st, lp.SCHED_FUSED, precision=prec)
    b = _run(st, lp.SCHED_SPLIT, precision=prec)
    assert a[3]["n_flagged"] > 0
    _same(a, b)


@pytest.mark.parametrize("prec", [lp.PREC_FP32, lp.PREC_FP64])
def test_work_queue_schedules_equal_the_launch_grid(prec):
    """The persistent kernels with warp work queues (query tiles, and the split
    fit's two kernels on the FP32 path) compute every particle with the same
    code as the one-warp-per-tile and one-thread-per-particle launches: the
    same state, flags and limiter values, bit for bit."""
    st = _cloud()
    a = _run(st, lp.SCHED_SPLIT, precision=prec)
    b = _run(st, lp.SCHED_SPLIT | lp.SCHED_QUEUE_FIT | lp.SCHED_QUEUE_QUERY, precision=prec)
    _same(a, b)


def _gate_threshold(st, params):
    """Median probability of the (untrained) network on the cloud's features:
    about half the particles fall below it."""
    ctx = lp.Context(_cfg(st))
    ctx.mlp_set_params(params)
    ps = lp.ParticleSet.from_state(st)
    feats = torch.empty((N, 8), dtype=torch.float32, device="cuda")
    ctx.step(ps, dt=1e-6, features=feats)
    p = ctx.mlp_infer(feats).cpu().numpy()
    ctx.close()
    return float(np.quantile(p, 0.5))


@pytest.mark.parametrize("audit", [0, 1])
def test_split_equals_fused_learned_estimator(audit):
    st = _cloud()
    params = lp.mlp_init_params(3)
    tau = _gate_threshold(st, params)
    kw = dict(estimator=lp.EST_MLP, mlp_tau_lo=tau, mlp_audit=audit)
    a = _run(st, lp.SCHED_FUSED, params=params, **kw)
    b = _run(st, lp.SCHED_SPLIT, params=params, **kw)
    skip = a[3]["n_mlp_skip"]
    assert 0.2 * 2 * N < skip < 0.8 * 2 * N, skip
    if audit:
        assert a[3]["n_mlp_miss"] > 0        # an untrained gate misses flags; the audit sees them
    _same(a, b)
    # the split kernels from work queues: a list of about half the particles
    c = _run(st, lp.SCHED_SPLIT | lp.SCHED_QUEUE_FIT, params=params, **kw)
    _same(a, c)


def test_default_schedule_follows_estimator():
    st = _cloud()
    c1 = lp.Context(_cfg(st))
    c2 = lp.Context(_cfg(st, estimator=lp.EST_MLP, mlp_tau_lo=0.1))
    assert c1.schedule() == lp.SCHED_FUSED
    assert c2.schedule() == lp.SCHED_SPLIT
    with pytest.raises(lp.LPError):
        c1.set_schedule(16)                  # no such schedule bit
    c1.close()
    c2.close()


def test_autotune_keeps_state_and_counters():
    st = _cloud()
    ref = _run(st, lp.SCHED_FUSED, steps=2)
    ctx = lp.Context(_cfg(st))
    ps = lp.ParticleSet.from_state(st)
    flag = torch.empty(N, dtype=torch.uint8, device="cuda")
    phi = torch.empty((N, 5), dtype=torch.float32, device="cuda")
    ctx.step(ps, dt=0.0, cfl=0.4, flag=flag, phi=phi)
    torch.cuda.synchronize()
    before = ps.to_state(N)
    s0 = ctx.stats()
    t = ctx.autotune(ps, dt=0.0, cfl=0.4, reps=2)
    assert all(v > 0 for v in t.values()), t
    fits = {lp.SCHED_FUSED: t["fit_fused"], lp.SCHED_SPLIT: t["fit_split"],
            lp.SCHED_SPLIT | lp.SCHED_QUEUE_FIT: t["fit_split_queue"]}
    queries = {0: t["query_tile"], lp.SCHED_QUERY_WARP: t["query_warp"], lp.SCHED_QUEUE_QUERY: t["query_tile_queue"]}
    want = min(fits, key=fits.get) | min(queries, key=queries.get)
    assert ctx.schedule() == want, (t, ctx.schedule())
    after = ps.to_state(N)
    for f in ("V", "P", "m", "id"):
        assert np.array_equal(before[f], after[f]), f
    for d in range(3):
        assert np.array_equal(before["x"][d], after["x"][d])
    s1 = ctx.stats()
    assert s0 == s1
    # the next step continues as if no tuning had happened
    ctx.step(ps, dt=0.0, cfl=0.4, flag=flag, phi=phi)
    torch.cuda.synchronize()
    got = (ps.to_state(N), flag.cpu().numpy(), phi.cpu().numpy(), ctx.stats())
    ctx.close()
    _same(ref, got)


def test_query_schedules_give_identical_lists():
    """Tiles (with the per-particle kernel for the particles they leave), one
    warp per particle for every particle, and tiles taken from a work queue by
    a persistent grid: the same lists, bit for bit."""
    st = _cloud()
    out = []
    for sched in (lp.SCHED_FUSED, lp.SCHED_QUERY_WARP, lp.SCHED_QUEUE_QUERY):
        ctx = lp.Context(_cfg(st))
        ctx.set_schedule(sched)
        ps = lp.ParticleSet.from_state(st)
        ctx.build_neighbors(ps)
        cnt, tot, idx, d2, keys = ctx.export_neighbors(N)
        out.append([a.cpu().numpy() for a in (cnt, tot, idx, d2, ps.id)])
        ctx.close()
    for other in out[1:]:
        for a, b in zip(out[0], other):
            assert np.array_equal(a, b)
