"""Parity at the benchmark's full size and launch configuration.

The 3D gas cloud with 2,000,000 particles (the workload bench.py times), the
same cloud with its tail beyond 4 sigma kept, and the jet-shaped snapshot with
8.0M are advanced one step on the GPU, under the schedule bench.py's
autotuner picks, with the CFL time step computed on the device.  The oracle
then evaluates, one particle at a time, the central derivatives (FP32 fit with
its correction pass), the neighbour lists, the new state and the rates of a
seeded sample of particles from the same full state, so the comparison is
element by element on those samples.  The 1M-particle jittered lattice of the
GFD workload is compared the same way, in FP32 and FP64, and with the analytic
derivatives.  Also: the Sod shock tube
run to t = 0.2 on the GPU's FP64 path converges to the exact Riemann solution
as closely as the oracle's own run does.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2206_11998_gb300 import inputs, lp
from tests import parity
from tests.gpu_util import ensure_built, normwise

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    oracle.build()


FULL = {
    # the workload bench.py times by default, the same cloud with its tail
    # beyond 4 sigma kept (a few far particles with two or three neighbours,
    # whose stencils degenerate), and the jet-shaped snapshot; all under the
    # schedule bench.py's autotuner picks (split fit, query tiles)
    "gas-cloud-2M": (lambda: inputs.gas_cloud_3d(2_000_000, seed=4), 5.0 / 3.0),
    "gas-cloud-2M-with-tail": (lambda: inputs.gas_cloud_3d(2_000_000, seed=4, r_max_sigma=0), 5.0 / 3.0),
    "jet-snapshot-8M": (lambda: inputs.jet_snapshot_3d(8_000_000, seed=10), inputs.JET_GAMMA),
}

FP32_GRAD_TOL = 1e-5      # the bars of test_gpu_parity.py (derived there)
FP32_HESS_TOL = 1e-3


def _samples(st, n, name):
    rng = np.random.default_rng(123)
    q = np.sort(rng.choice(n, 400, replace=False))
    # extremes of the distribution too: the outermost particles have the largest radii
    # (the cloud), the largest specific volumes sit by the density jump (the jet)
    r2 = st["x"][0] ** 2 + st["x"][1] ** 2 + st["x"][2] ** 2
    extra = [np.argsort(r2)[-20:], np.argsort(r2)[:20], np.argsort(st["V"])[-20:]]
    if name.startswith("jet"):
        # the jet is uniform inside and outside, and no ambient particle lies
        # within half its spacing of the jet's surface (radius 1 about the z
        # axis, 0 <= z <= 12), so a jet particle's neighbours are all jet
        # particles: what changes in a step are the ambient particles whose
        # radius reaches the jet.  120 of them are drawn from the initial state.
        rc = np.sqrt(st["x"][0] ** 2 + st["x"][1] ** 2)
        z = st["x"][2]
        out = np.maximum(rc - 1.0, 0.0)
        dist = np.where(z <= 12.0, out, np.hypot(out, z - 12.0))
        R = 2.2 * np.cbrt(st["m"] * st["V"])
        near = np.nonzero((st["V"] > 10.0 * st["V"].min()) & (dist < R))[0]
        extra.append(rng.choice(near, min(120, len(near)), replace=False))
    return np.unique(np.concatenate([q] + extra))


@pytest.mark.parametrize("name", list(FULL))
def test_full_size_sampled_parity(name):
    make, gamma = FULL[name]
    st = make()
    n = st["V"].shape[0]
    sref = inputs.field_scales(st)
    cfg = lp.make_config(3, n, precision=lp.PREC_FP32, kappa=2.2, k_max=64, k_side=8, gamma=gamma,
                         limiter=lp.LIM_FLAGGED, s_ref=sref)
    ctx = lp.Context(cfg)
    ctx.set_schedule(lp.SCHED_SPLIT)
    ps = lp.ParticleSet.from_state(st)
    q = _samples(st, n, name)
    ocfg = oracle.make_config(3, gamma=gamma, kappa=2.2, k_max=64, k_side=8, limiter=oracle.LIM_FLAGGED,
                              s_ref=sref)
    oidx, ocnt, otot, od2 = oracle.neighbors(ocfg, st["x"], st["V"], st["m"], st["id"], query=q)

    # central derivatives of the five fields (lp_gfd_derivs, FP32 with the
    # default correction pass) on the lists of this state
    ctx.build_neighbors(ps)
    ids = ps.id.cpu().numpy().astype(np.int64)
    pos = np.empty(n, np.int64)
    pos[ids] = np.arange(n)
    status = torch.zeros(n, dtype=torch.int32, device="cuda")
    fields = [ps.V, ps.u[0], ps.u[1], ps.u[2], ps.P]
    gd = ctx.gfd_derivs(ps, fields, lp.OUT_F64, status=status).cpu().numpy()[:, pos[q], :]
    gst = status.cpu().numpy()[pos[q]]
    ofields = [st["V"], st["u"][0], st["u"][1], st["u"][2], st["P"]]
    od, ost = oracle.gfd_central(ocfg, st["x"], ofields, ocnt, oidx, query=q)
    # the same fit kind (second order, first-order fallback, none) for every sample
    assert np.array_equal(gst & 3, ost & 3), np.nonzero((gst & 3) != (ost & 3))
    e_g = max(normwise(gd[f][:, u], od[f][:, u]) for f in range(5) for u in range(3))
    e_h = max(normwise(gd[f][:, u], od[f][:, u]) for f in range(5) for u in range(3, 9))
    print("%s: %d samples, FP64 redo %d, gradient error %.2e, second-derivative error %.2e"
          % (name, len(q), int(((gst & 8) != 0).sum()), e_g, e_h))
    assert e_g < FP32_GRAD_TOL
    assert e_h < FP32_HESS_TOL

    # one step with the CFL step computed on the device
    phi = torch.empty((n, 5), dtype=torch.float32, device="cuda")
    flag = torch.empty(n, dtype=torch.uint8, device="cuda")
    ctx.step(ps, dt=0.0, cfl=0.4, phi=phi, flag=flag)
    torch.cuda.synchronize()
    dt = ctx.stats()["dt"]
    cnt, tot, idx, d2, keys = ctx.export_neighbors(n)
    ids = ps.id.cpu().numpy().astype(np.int64)
    pos[ids] = np.arange(n)
    # neighbour lists of the samples, bit-exact
    cnt = cnt.cpu().numpy(); tot = tot.cpu().numpy(); idx = idx.cpu().numpy(); d2 = d2.cpu().numpy()
    for r, pid in enumerate(q):
        i = pos[pid]
        assert np.array_equal(ids[idx[i, :cnt[i]]], oidx[r, :ocnt[r]]), pid
        assert tot[i] == otot[r] and d2[i] == od2[r]
    # new state of the samples, with the GPU's phi forced where a decision
    # differs inside the ambiguity band
    o = oracle.step(ocfg, st, dt, query=q)
    gphi = phi.cpu().numpy()[pos[q]]
    gflag = flag.cpu().numpy()[pos[q]]
    o, ndiff = parity.resolve(ocfg, st, q, lp.PREC_FP32, gflag, gphi, o, dt, 6)
    g = {"V": ps.V.cpu().numpy()[pos[q]], "P": ps.P.cpu().numpy()[pos[q]],
         "u": [ps.u[k].cpu().numpy()[pos[q]] for k in range(3)], "x": [ps.x[k].cpu().numpy()[pos[q]] for k in range(3)]}
    s0 = {"V": st["V"][q], "P": st["P"][q], "u": [st["u"][k][q] for k in range(3)]}
    errs, rates = parity.field_and_rate_errors(3, s0, g, o, dt)
    changed = int((np.abs(g["P"] - s0["P"]) > 0).sum())
    print("%s: %d of %d samples changed; ambiguous %d; field errors %s; rate errors %s"
          % (name, changed, len(q), ndiff, errs, rates))
    assert changed >= min(30, len(q) // 2)
    for k in ("V", "u0", "u1", "u2", "P"):
        assert errs[k] < 1e-5, (k, errs)
        assert rates[k] < RATE_TOL[k[0]], (k, rates)
    # the mover, x + dt (u^n + u^{n+1}) / 2, carries the new velocity's error
    # (FP32: below 1e-5 of max |u^{n+1}|) into the position: dt / 2 times it,
    # on top of the FP64 rounding of x
    umax = max(np.abs(o["u"][k]).max() for k in range(3))
    for k in range(3):
        bound = 0.5 * dt * 1e-5 * umax + 1e-13 * np.abs(o["x"][k]).max()
        assert np.abs(g["x"][k] - o["x"][k]).max() <= bound, (k, errs["x%d" % k], bound)
    ctx.close()


RATE_TOL = {"V": 1e-4, "u": 1e-4, "P": 1e-4}     # FP32 bars of test_gpu_parity.py (derived there)


def test_gfd_lattice_1M_fp32_fp64_analytic():
    """The GFD kernel alone on its own workload at full size: 1M particles on
    a jittered cubic lattice (h = 1/100, jitter 0.2 h), fixed radius 2.2 h
    (about 43 neighbours), one quadratic field plus N(0, 1e-6^2) noise.  FP32
    with the correction pass and FP64 on the GPU against the oracle on sampled
    particles, and both against the analytic derivatives of the noise-free
    quadratic (whose distance is set by the noise, ~1e-6 / h per gradient)."""
    n_side, h = 100, 0.01
    x, fields, coeffs = inputs.gfd_lattice_workload(n_side, h, 1e-6)
    n = x[0].shape[0]
    st = {"x": x, "V": np.ones(n), "u": [np.zeros(n)] * 3, "P": np.ones(n), "m": np.ones(n),
          "id": np.arange(n, dtype=np.uint32), "n_fluid": n}
    rng = np.random.default_rng(7)
    q = np.sort(rng.choice(n, 500, replace=False))
    ocfg = oracle.make_config(3, radius_mode=oracle.RADIUS_FIXED, radius=2.2 * h, k_max=64)
    oidx, ocnt, _, _ = oracle.neighbors(ocfg, x, st["V"], st["m"], st["id"], query=q)
    od, _ = oracle.gfd_central(ocfg, x, fields, ocnt, oidx, query=q)
    c, g0, H = coeffs[0]
    X = np.stack([a[q] for a in x])
    grad = (g0[:, None] + H @ X).T
    out = {}
    for prec in (lp.PREC_FP32, lp.PREC_FP64):
        cfg = lp.make_config(3, n, precision=prec, radius_mode=lp.RADIUS_FIXED, radius=2.2 * h, k_max=64)
        ctx = lp.Context(cfg)
        ps = lp.ParticleSet.from_state(st)
        ctx.build_neighbors(ps)
        ids = ps.id.cpu().numpy().astype(np.int64)
        pos = np.empty(n, np.int64)
        pos[ids] = np.arange(n)
        f = torch.as_tensor(fields[0][ids], device="cuda")
        d = ctx.gfd_derivs(ps, [f], lp.OUT_F64).cpu().numpy()[0][pos[q]]
        ctx.close()
        out[prec] = d
    e32 = max(normwise(out[lp.PREC_FP32][:, u], od[0][:, u]) for u in range(3))
    e32h = max(normwise(out[lp.PREC_FP32][:, u], od[0][:, u]) for u in range(3, 9))
    e64 = max(normwise(out[lp.PREC_FP64][:, u], od[0][:, u]) for u in range(9))
    a32 = normwise(out[lp.PREC_FP32][:, :3], grad)
    a64 = normwise(out[lp.PREC_FP64][:, :3], grad)
    ao = normwise(od[0][:, :3], grad)
    print("1M lattice: FP32 vs oracle grad %.2e hess %.2e; FP64 vs oracle %.2e; vs analytic: oracle %.2e "
          "FP32 %.2e FP64 %.2e" % (e32, e32h, e64, ao, a32, a64))
    assert e32 < FP32_GRAD_TOL and e32h < FP32_HESS_TOL
    assert e64 < 1e-11
    # the noise sets the distance to the analytic gradient (the oracle's own:
    # ~2e-4); the GPU forms are that far too, FP32 within its bar of it
    assert ao < 1e-3
    assert abs(a32 - ao) < FP32_GRAD_TOL and abs(a64 - ao) < 1e-10


def _sod_l1(state, n_fluid, t):
    f = state["id"] < n_fluid
    x = state["x"][0][f]
    r, u, p = oracle.riemann_exact(1.4, (1, 0, 1), (0.125, 0, 0.1), 0.5, t, x)
    return (np.mean(np.abs(1 / state["V"][f] - r)), np.mean(np.abs(state["u"][0][f] - u)),
            np.mean(np.abs(state["P"][f] - p)))


def test_sod_fp64_run_to_t02_converges():
    golden = {}
    path = os.path.join(os.path.dirname(__file__), "golden", "sod_oracle_l1.txt")
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            golden[k] = float(v)
    st = inputs.sod_1d(889, 111)
    n = st["V"].shape[0]
    cfg = lp.make_config(1, n, precision=lp.PREC_FP64, radius_mode=lp.RADIUS_KSIDE, k_max=8, k_per_side=4,
                         k_side=1, gamma=1.4, s_ref=inputs.field_scales(st), n_fluid=st["n_fluid"])
    ctx = lp.Context(cfg)
    ps = lp.ParticleSet.from_state(st)
    t, dt = 0.0, 0.0
    while dt == 0.0 or 0.2 - t > 2.0 * dt:
        ctx.step(ps, dt=0.0, cfl=0.4)     # CFL step computed on the device
        dt = ctx.stats()["dt"]
        t += dt
    k = int(np.ceil((0.2 - t) / dt))      # land on t = 0.2 with k equal steps <= the CFL step
    for _ in range(k):
        ctx.step(ps, dt=(0.2 - t) / k if _ == 0 else h, cfl=0.4)
        h = (0.2 - t) / k
    t = 0.2
    g = ps.to_state(st["n_fluid"])
    e = _sod_l1(g, st["n_fluid"], t)
    # the GPU's errors match the oracle's own run to within 10 %, and stay small
    assert e[0] < 1.1 * golden["rho_l1"] + 1e-4
    assert e[1] < 1.1 * golden["u_l1"] + 1e-4
    assert e[2] < 1.1 * golden["p_l1"] + 1e-4
    ctx.close()
