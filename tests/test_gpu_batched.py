"""Batched steps of many independent simulations (lp_step_batched).

Each simulation advanced inside one batched call must equal, bit for bit (by
particle id), the same simulation advanced alone: the simulations share one
sort, one set of cell tables and one launch per phase, but neither their
neighbour lists (exact, in (d^2, id) order) nor their per-simulation CFL steps
depend on the other simulations.  One batched step is also compared with the
FP64 oracle per simulation.
"""
import numpy as np
import pytest

import oracle
from paper_2206_11998_gb300 import inputs, lp
from tests.gpu_util import by_id, ensure_built, normwise

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    oracle.build()


def _ensemble(sizes, seed0=50):
    sims = [inputs.kh_2d(int(n), 0.01 + 0.01 * k, seed=seed0 + k) for k, n in enumerate(sizes)]
    return sims


def _concat(sims):
    keys = ["V", "P", "m"]
    st = {k: np.concatenate([s[k] for s in sims]) for k in keys}
    st["x"] = [np.concatenate([s["x"][a] for s in sims]) for a in range(2)]
    st["u"] = [np.concatenate([s["u"][a] for s in sims]) for a in range(2)]
    n = st["V"].shape[0]
    st["id"] = np.arange(n, dtype=np.uint32)
    st["n_fluid"] = n
    offs = np.concatenate([[0], np.cumsum([s["V"].shape[0] for s in sims])]).astype(np.int64)
    return st, offs


def _cfg(n, prec, nsim):
    return lp.make_config(2, n, precision=prec, kappa=2.2, k_max=40, gamma=1.4, periodic=(1, 1, 0),
                          box_lo=(0, 0, 0), box_hi=(1, 1, 1), s_ref=(1.0, 0.5, 0.5, 2.5), max_sims=nsim)


@pytest.mark.parametrize("prec", [lp.PREC_FP32, lp.PREC_FP64])
def test_batched_equals_each_simulation_alone(prec):
    sizes = [3001, 5200, 1777, 4096, 2500, 6003]
    sims = _ensemble(sizes)
    st, offs = _concat(sims)
    n = st["V"].shape[0]
    ctx = lp.Context(_cfg(n, prec, len(sims)))
    ps = lp.ParticleSet.from_state(st)
    offs_d = torch.as_tensor(offs, device="cuda")
    t = torch.zeros(len(sims), dtype=torch.float64, device="cuda")
    for _ in range(3):
        ctx.step_batched(ps, offs_d, len(sims), dt=0.0, cfl=0.4, t=t)
    torch.cuda.synchronize()
    g = ps.to_state(n)
    ids = g["id"].astype(np.int64)
    # every simulation stays at its offsets
    for k in range(len(sims)):
        seg = ids[offs[k]:offs[k + 1]]
        assert seg.min() == offs[k] and seg.max() == offs[k + 1] - 1
    tb = t.cpu().numpy()
    for k, sim in enumerate(sims):
        nk = sim["V"].shape[0]
        c1 = lp.Context(_cfg(nk, prec, 1))
        p1 = lp.ParticleSet.from_state(sim)
        t1 = torch.zeros(1, dtype=torch.float64, device="cuda")
        for _ in range(3):
            c1.step(p1, dt=0.0, cfl=0.4, t=t1)
        a = p1.to_state(nk)
        ia = a["id"].astype(np.int64)
        sl = slice(offs[k], offs[k + 1])
        ib = ids[sl] - offs[k]
        for f in ("V", "P"):
            assert np.array_equal(by_id(ia, a[f]), by_id(ib, g[f][sl])), (k, f)
        for d in range(2):
            assert np.array_equal(by_id(ia, a["u"][d]), by_id(ib, g["u"][d][sl])), (k, d)
            assert np.array_equal(by_id(ia, a["x"][d]), by_id(ib, g["x"][d][sl])), (k, d)
        assert float(t1.cpu()[0]) == tb[k]
        c1.close()
    ctx.close()


def test_batched_step_matches_oracle_per_simulation():
    sizes = [2500, 4001, 3333]
    sims = _ensemble(sizes, seed0=70)
    st, offs = _concat(sims)
    n = st["V"].shape[0]
    ctx = lp.Context(_cfg(n, lp.PREC_FP64, len(sims)))
    ps = lp.ParticleSet.from_state(st)
    offs_d = torch.as_tensor(offs, device="cuda")
    ctx.step_batched(ps, offs_d, len(sims), dt=1e-3, cfl=0.4)
    g = ps.to_state(n)
    ids = g["id"].astype(np.int64)
    for k, sim in enumerate(sims):
        ocfg = oracle.make_config(2, gamma=1.4, kappa=2.2, k_max=40, periodic=(1, 1, 0), box_lo=(0, 0, 0),
                                  box_hi=(1, 1, 1), s_ref=(1.0, 0.5, 0.5, 2.5))
        o = oracle.step(ocfg, sim, 1e-3)
        sl = slice(offs[k], offs[k + 1])
        ib = ids[sl] - offs[k]
        assert normwise(by_id(ib, g["P"][sl]), o["P"]) < 1e-12
        assert normwise(by_id(ib, g["V"][sl]), o["V"]) < 1e-12
        for d in range(2):
            assert normwise(by_id(ib, g["u"][d][sl]), o["u"][d]) < 1e-12
    ctx.close()


@pytest.mark.parametrize("queue", [False, True])
def test_graph_replay_equals_eager_steps(queue):
    """A step captured into a CUDA graph and replayed equals the same steps run
    eagerly, bit for bit; with queue, the graph replays the persistent kernels
    that take their work from warp work queues (tiles of the query, particles
    and list entries of the split fit), whose counters the graph itself resets."""
    sims = _ensemble([2000, 3500, 2800], seed0=90)
    st, offs = _concat(sims)
    n = st["V"].shape[0]
    outs = []
    for mode in ("eager", "graph"):
        ctx = lp.Context(_cfg(n, lp.PREC_FP32, len(sims)))
        if queue and mode == "graph":
            ctx.set_schedule(lp.SCHED_SPLIT | lp.SCHED_QUEUE_FIT | lp.SCHED_QUEUE_QUERY)
        ps = lp.ParticleSet.from_state(st)
        offs_d = torch.as_tensor(offs, device="cuda")
        t = torch.zeros(len(sims), dtype=torch.float64, device="cuda")
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            ctx.step_batched(ps, offs_d, len(sims), dt=0.0, cfl=0.4, t=t, stream=s)
            if mode == "eager":
                for _ in range(4):
                    ctx.step_batched(ps, offs_d, len(sims), dt=0.0, cfl=0.4, t=t, stream=s)
            else:
                ctx.graph_capture(ps, offs_d, len(sims), dt=0.0, cfl=0.4, t=t, stream=s)
                for _ in range(4):
                    ctx.graph_launch(stream=s)
            s.synchronize()
        g = ps.to_state(n)
        outs.append((g, t.cpu().numpy(), ctx.stats()["steps"]))
        ctx.close()
    (a, ta, na), (b, tb, nb) = outs
    assert na == nb == 5
    assert np.array_equal(ta, tb)
    assert np.array_equal(a["id"], b["id"])
    for f in ("V", "P"):
        assert np.array_equal(a[f], b[f])
    for d in range(2):
        assert np.array_equal(a["x"][d], b["x"][d]) and np.array_equal(a["u"][d], b["u"][d])
