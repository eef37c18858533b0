"""Reservoir inflow through a nozzle inlet (Sec. 4, the inlet boundary
condition of the supersonic-jet simulations; Sec. 2.2 step 1: inflow
boundaries generate particles) on the GPU, with capacity growth.

A jet grows from an ambient gas at rest through a Mach-3 reservoir inlet.  At
every call of lp_inflow, after a step:
  - P_inf is the mean pressure of the fluid particles near the inlet (checked
    against the state the call saw), and (rho_inf, u_inf) are the oracle's
    reservoir inflow state for it;
  - exactly `layers` whole layers of npat particles were appended, each with
    the injected mass and the inflow state, inside the inlet disk and past the
    inlet plane, with ids not seen before; the reservoir ghosts behind the
    inlet carry the inflow state;
  - mass is conserved exactly: every particle keeps its mass, and the total
    grows by the injected particles' mass.
The step itself, with the ghosts as frozen boundary particles, is compared
with the oracle on sampled particles by the inlet.
"""
import numpy as np
import pytest

import oracle
from paper_2206_11998_gb300 import inputs, lp
from tests import parity
from tests.gpu_util import ensure_built

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GHOST_ID = 2 ** 31
N_FLUID = 2 ** 31


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    oracle.build()


def _setup(h, capacity):
    st, q = inputs.jet_inflow_3d(h)
    inlet = lp.make_inlet(q["center"], q["axis"], q["radius"], q["spacing"], q["mass"], q["P_res"], q["rho_res"],
                          q["sample_depth"], ghost_layers=q["ghost_layers"], first_id=st["V"].shape[0],
                          ghost_id=GHOST_ID)
    cfg = lp.make_config(3, capacity, kappa=2.2, k_max=64, gamma=inputs.JET_GAMMA, n_fluid=N_FLUID,
                         s_ref=(1.0, 1.0, 1.0, 3.5, 1.0))
    return st, q, inlet, cfg


def _near_inlet(s, q):
    rc2 = s["x"][0] ** 2 + s["x"][1] ** 2
    return (s["id"] < N_FLUID) & (s["x"][2] >= 0.0) & (s["x"][2] <= q["sample_depth"]) & (rc2 <= q["radius"] ** 2)


def test_inflow_state_layers_and_mass():
    h = 0.1
    st, q, inlet, cfg = _setup(h, 200_000)
    ctx = lp.Context(cfg)
    ps = lp.ParticleSet.with_capacity(st, 200_000)
    g = inputs.JET_GAMMA
    seen = set(st["id"].tolist())
    mass0 = float(st["m"].sum())
    info = ctx.inflow(ps, inlet)                       # first call: the ghosts, no fluid yet
    assert info["layers"] == 0 and abs(info["P_inf"] - q["P_res"]) < 1e-15 * q["P_res"]
    npat = info["npat"]
    assert ps.n == st["V"].shape[0] + q["ghost_layers"] * npat
    total_layers = 0
    hz_prev = info["h_z"]
    for step in range(40):
        ctx.step(ps, dt=0.0, cfl=0.4)
        dt = ctx.stats()["dt"]
        before = ps.to_state()
        mass_before = float(before["m"].sum())
        info = ctx.inflow(ps, inlet)
        after = ps.to_state()
        # P_inf: the mean pressure near the inlet of the state the call saw
        near = _near_inlet(before, q)
        assert info["sampled"] == int(near.sum())
        if near.any():
            assert abs(info["P_inf"] - before["P"][near].mean()) <= 1e-12 * info["P_inf"]
        rho, u = oracle.inflow_state(g, q["P_res"], q["rho_res"], info["P_inf"])
        assert abs(info["rho_inf"] - rho) <= 1e-13 * rho and abs(info["u_inf"] - u) <= 1e-13 * max(u, 1e-300)
        assert abs(info["h_z"] - q["mass"] / (rho * h * h)) <= 1e-13 * info["h_z"]
        # whole layers, appended after the particles the call saw
        nl = info["layers"]
        total_layers += nl
        assert info["layers_total"] == total_layers
        assert after["V"].shape[0] == before["V"].shape[0] + nl * npat
        assert np.array_equal(after["id"][:before["V"].shape[0]], before["id"])
        new = slice(before["V"].shape[0], None)
        ids = after["id"][new]
        assert len(set(ids.tolist()) & seen) == 0 and len(set(ids.tolist())) == ids.shape[0]
        seen.update(ids.tolist())
        if nl:
            z = after["x"][2][new]
            assert z.min() >= 0.0 and z.max() < u * dt + max(hz_prev, info["h_z"]) * (1 + 1e-12)
            rc = np.sqrt(after["x"][0][new] ** 2 + after["x"][1][new] ** 2)
            assert rc.max() <= q["radius"] + h
            assert np.all(after["P"][new] == info["P_inf"]) and np.all(after["u"][2][new] == info["u_inf"])
            assert np.all(after["u"][0][new] == 0.0) and np.all(after["V"][new] == 1.0 / info["rho_inf"])
        # the ghosts: behind the inlet, with the inflow state
        gh = after["id"] >= GHOST_ID
        assert gh.sum() == q["ghost_layers"] * npat
        assert np.all(after["x"][2][gh] < info["travel"]) and np.all(after["P"][gh] == info["P_inf"])
        hz_prev = info["h_z"]
        # mass: unchanged per particle, grown by the injected particles
        assert float(after["m"].sum()) == pytest.approx(mass_before + nl * npat * q["mass"], rel=1e-14)
    assert total_layers > 5, total_layers
    fluid = ps.to_state()
    f = fluid["id"] < N_FLUID
    assert float(fluid["m"][f].sum()) == pytest.approx(mass0 + total_layers * npat * q["mass"], rel=1e-13)
    print("inflow: %d layers of %d in 40 steps, P_inf %.3g, u_inf %.3g (Mach %.2f), n %d"
          % (total_layers, npat, info["P_inf"], info["u_inf"], info["u_inf"] / info["c_inf"], ps.n))
    ctx.close()


def test_inflow_step_matches_oracle_by_the_inlet():
    """After 20 steps of growth, one more step against the oracle on the
    particles by the inlet (fluid, ghosts frozen) and a random sample."""
    h = 0.1
    st, q, inlet, cfg = _setup(h, 200_000)
    ctx = lp.Context(cfg)
    ps = lp.ParticleSet.with_capacity(st, 200_000)
    ctx.inflow(ps, inlet)
    for _ in range(20):
        ctx.step(ps, dt=0.0, cfl=0.4)
        ctx.inflow(ps, inlet)
    s0 = ps.to_state()
    n = s0["V"].shape[0]
    phi = torch.empty((ps.capacity, 5), dtype=torch.float32, device="cuda")
    flag = torch.empty(ps.capacity, dtype=torch.uint8, device="cuda")
    ctx.step(ps, dt=0.0, cfl=0.4, phi=phi, flag=flag)
    dt = ctx.stats()["dt"]
    g1 = ps.to_state()
    order = np.argsort(g1["id"])
    sorted_ids = g1["id"][order]
    where = lambda ids: order[np.searchsorted(sorted_ids, ids)]      # id -> position after the step
    rc2 = s0["x"][0] ** 2 + s0["x"][1] ** 2
    by_inlet = np.nonzero((s0["id"] < N_FLUID) & (s0["x"][2] < 4 * h) & (rc2 < 1.2))[0]
    rng = np.random.default_rng(5)
    q_idx = np.unique(np.concatenate([rng.choice(by_inlet, min(150, len(by_inlet)), replace=False),
                                      rng.choice(n, 150, replace=False)]))
    ocfg = oracle.make_config(3, gamma=inputs.JET_GAMMA, kappa=2.2, k_max=64, k_side=8, limiter=oracle.LIM_FLAGGED,
                              s_ref=(1.0, 1.0, 1.0, 3.5, 1.0), n_fluid=N_FLUID)
    o = oracle.step(ocfg, s0, dt, query=q_idx)
    gpos = where(s0["id"][q_idx])
    assert np.array_equal(g1["id"][gpos], s0["id"][q_idx])
    gphi = phi.cpu().numpy()[gpos]
    gflag = flag.cpu().numpy()[gpos]
    o, ndiff = parity.resolve(ocfg, s0, q_idx, lp.PREC_FP32, gflag, gphi, o, dt, 6)
    g = {"V": g1["V"][gpos], "P": g1["P"][gpos], "u": [g1["u"][k][gpos] for k in range(3)],
         "x": [g1["x"][k][gpos] for k in range(3)]}
    sq = {"V": s0["V"][q_idx], "P": s0["P"][q_idx], "u": [s0["u"][k][q_idx] for k in range(3)]}
    errs, rates = parity.field_and_rate_errors(3, sq, g, o, dt)
    print("inflow step vs oracle: %d samples (%d by the inlet), ambiguous %d; fields %s" % (len(q_idx), len(by_inlet),
                                                                                          ndiff, errs))
    for k in ("V", "u0", "u1", "u2", "P"):
        assert errs[k] < 1e-5, (k, errs)
    ctx.close()


def test_capacity_growth_with_reserve():
    """A context and arrays sized tight: lp_inflow refuses to overflow them,
    leaves the state where it was, and after growing both (ParticleSet.grown,
    lp_reserve) the same call succeeds and the run goes on."""
    h = 0.1
    st, q, inlet, cfg0 = _setup(h, 1)
    n0 = st["V"].shape[0]
    cap = n0 + 3 * 400 + 200
    _, _, _, cfg = _setup(h, cap)
    ctx = lp.Context(cfg)
    ps = lp.ParticleSet.with_capacity(st, cap)
    ctx.inflow(ps, inlet)
    grew = 0
    for _ in range(60):
        ctx.step(ps, dt=0.0, cfl=0.4)
        try:
            ctx.inflow(ps, inlet)
        except lp.LPError as e:
            assert e.code == lp.ERR_CAPACITY
            n_before = ps.n
            ps = ps.grown(ps.capacity + 700)            # room for two more layers
            ctx.reserve(ps.capacity)
            info = ctx.inflow(ps, inlet)
            assert info["layers"] > 0 and ps.n == n_before + info["layers"] * info["npat"]
            grew += 1
    assert grew >= 2, grew
    ctx.step(ps, dt=0.0, cfl=0.4)
    s = ctx.stats()
    assert s["n_nonfinite"] >= 0
    ctx.close()


def test_outflow_removes_particles_outside_the_box_in_order():
    """lp_remove_outside keeps the particles inside the box, in their order,
    with their state; the lists are stale until the next build."""
    st = inputs.gas_cloud_3d(50_000, seed=3)
    n = st["V"].shape[0]
    cfg = lp.make_config(3, n, kappa=2.2, k_max=64, gamma=5.0 / 3.0, s_ref=inputs.field_scales(st))
    ctx = lp.Context(cfg)
    ps = lp.ParticleSet.with_capacity(st, n)
    ctx.step(ps, dt=0.0, cfl=0.4)
    before = ps.to_state()
    lo, hi = (-0.3, -0.2, -10.0), (0.25, 10.0, 0.3)
    keep = np.ones(n, bool)
    for k in range(3):
        keep &= (before["x"][k] >= lo[k]) & (before["x"][k] <= hi[k])
    removed = ctx.remove_outside(ps, lo, hi)
    after = ps.to_state()
    assert removed == n - keep.sum() and removed > 0
    for f in ("V", "P", "m", "id"):
        assert np.array_equal(after[f], before[f][keep]), f
    for k in range(3):
        assert np.array_equal(after["x"][k], before["x"][k][keep])
        assert np.array_equal(after["u"][k], before["u"][k][keep])
    with pytest.raises(lp.LPError):
        ctx.export_neighbors(n)
    ctx.step(ps, dt=0.0, cfl=0.4)                     # a build makes them current again
    ctx.export_neighbors(ps.n)
    ctx.close()
