"""GPU parity of the CUDA path (through the C ABI) with the FP64 oracle.

Integer and index results (Morton keys, sort order, neighbour lists, counts) are
bit-exact.  Floating-point results are compared normwise per field,
max|gpu - oracle| / max|oracle|:
  fields after one step: FP64 path <= 1e-12, FP32 path <= 1e-5 (the targets);
  derivative components: the bounds derived from the arithmetic next to
  FP64_DERIV_TOL / FP32_GRAD_TOL / FP32_HESS_TOL below.
Discontinuous estimator decisions (r near 3/2, one-sided derivatives near a
sign change) may legitimately differ at round-off; such particles are listed,
checked to be within the ambiguity band, and the oracle is re-run with the
GPU's decision for them.
"""
import numpy as np
import pytest

import oracle
from paper_2206_11998_gb300 import inputs, lp
from tests import parity
from tests.gpu_util import by_id, ensure_built, gpu_neighbor_ids, normwise, state_by_id

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    oracle.build()


def _oracle_cfg(lcfg, n_fluid=2**62):
    return oracle.make_config(
        lcfg.dim, gamma=lcfg.gamma, radius_mode=lcfg.radius_mode, radius=lcfg.radius, kappa=lcfg.kappa,
        k_max=lcfg.k_max, k_side=lcfg.k_side, k_per_side=lcfg.k_per_side, limiter=lcfg.limiter,
        flat_eps=lcfg.flat_eps, active_frac=lcfg.active_frac, s_ref=list(lcfg.s_ref),
        periodic=list(lcfg.periodic), box_lo=list(lcfg.box_lo), box_hi=list(lcfg.box_hi),
        rank_tol=1e-12, n_fluid=n_fluid, select=lcfg.select)


def _check_lists(ctx, ps, st, ocfg):
    ids, lists, tot, d2, keys = gpu_neighbor_ids(ctx, ps)
    oidx, ocnt, otot, od2 = oracle.neighbors(ocfg, st["x"], st["V"], st["m"], st["id"])
    bad = 0
    for i, pid in enumerate(ids):
        ref = oidx[pid, :ocnt[pid]]
        if not (np.array_equal(lists[i], ref) and tot[i] == otot[pid] and d2[i] == od2[pid]):
            bad += 1
    assert bad == 0, "%d of %d lists differ" % (bad, len(ids))
    return ids, keys


CASES_NB = {
    "3d-fixed-lattice": lambda: (inputs.gfd_lattice_workload(21, 1.0 / 21, 0.0)[0], "fixed3"),
    "3d-volume-cloud": lambda: (inputs.gas_cloud_3d(20_037, seed=8), "vol3"),
    "2d-periodic-kh": lambda: (inputs.kh_2d(7_001, 0.03, seed=5), "kh2"),
    "1d-sod": lambda: (inputs.sod_1d(889, 111), "sod1"),
    # density contrast 1e3: ambient radii ~10x the jet's, lists truncated at k_max
    "3d-jet-snapshot": lambda: (inputs.jet_snapshot_3d(30_000), "vol3"),
}


def _case_state(name):
    obj, kind = CASES_NB[name]()
    if kind == "fixed3":
        x = obj
        n = x[0].shape[0]
        st = {"x": x, "V": np.ones(n), "u": [np.zeros(n)] * 3, "P": np.ones(n), "m": np.ones(n),
              "id": np.arange(n, dtype=np.uint32), "n_fluid": n}
        cfg = lp.make_config(3, n, radius_mode=lp.RADIUS_FIXED, radius=2.2 / 21, k_max=64)
    elif kind == "vol3":
        st = obj
        cfg = lp.make_config(3, st["V"].shape[0], radius_mode=lp.RADIUS_VOLUME, kappa=2.2, k_max=64)
    elif kind == "kh2":
        st = obj
        cfg = lp.make_config(2, st["V"].shape[0], radius_mode=lp.RADIUS_VOLUME, kappa=2.2, k_max=40,
                             periodic=(1, 1, 0), box_lo=(0, 0, 0), box_hi=(1, 1, 1))
    else:
        st = obj
        cfg = lp.make_config(1, st["V"].shape[0], radius_mode=lp.RADIUS_KSIDE, k_max=8, k_per_side=4,
                             k_side=1, n_fluid=st["n_fluid"])
    return st, cfg


@pytest.mark.parametrize("name", list(CASES_NB))
def test_neighbor_lists_bit_exact(name):
    st, cfg = _case_state(name)
    ctx = lp.Context(cfg)
    ps = lp.ParticleSet.from_state(st)
    ctx.build_neighbors(ps)
    torch.cuda.synchronize()
    ids, keys = _check_lists(ctx, ps, st, _oracle_cfg(cfg))
    # the permuted arrays carry their particles
    for k in range(len(st["x"])):
        assert np.array_equal(ps.x[k].cpu().numpy(), st["x"][k][ids])
    assert np.array_equal(ps.m.cpu().numpy(), st["m"][ids])
    if cfg.dim > 1:
        # Morton keys equal the oracle's definition on the GPU's cube, and the
        # order is the stable sort by the key's cell bits (ties keep input order)
        g = ctx.grid_info()
        okeys = oracle.morton_keys(st["x"], g[:cfg.dim], g[3], 21)
        assert np.array_equal(keys, okeys[ids])
        # the sort orders by the cell bits down to table level 9 (3D) or 13
        # (2D), in whole 9-bit digits
        top = cfg.dim * 21
        lo_bit = top - 9 * ((cfg.dim * (9 if cfg.dim == 3 else 13) + 8) // 9)
        order = np.lexsort((np.arange(len(okeys)), okeys >> np.uint64(max(lo_bit, 0))))
        assert np.array_equal(ids, order)
    ctx.close()


def test_neighbor_overflow_truncates_exactly():
    # dense core with a small capacity: most lists truncated at k_max
    st = inputs.gas_cloud_3d(12_000, seed=9)
    cfg = lp.make_config(3, 12_000, radius_mode=lp.RADIUS_VOLUME, kappa=3.0, k_max=24)
    ctx = lp.Context(cfg)
    ps = lp.ParticleSet.from_state(st)
    ctx.build_neighbors(ps)
    torch.cuda.synchronize()
    _check_lists(ctx, ps, st, _oracle_cfg(cfg))
    s = ctx.stats()
    assert s["n_overflow"] > 6000
    # more than 64 in reach: those lists come from the warp-per-particle kernel
    assert s["n_query_fallback"] > 1000
    ctx.close()


def _stencil_tail_count(st, idx, cnt, k_side):
    """Particles whose one-sided stencils (the first k_side list members on each
    side of each axis, Sec. 2.1) take a member at list position 64 or later."""
    x = np.stack(st["x"], 1)
    K = idx.shape[1]
    valid = np.arange(K)[None, :] < cnt[:, None]
    off = x[np.where(valid, idx, 0)] - x[:, None, :]
    tail = np.zeros(x.shape[0], bool)
    for k in range(x.shape[1]):
        for sg in (1.0, -1.0):
            mem = valid & (np.sign(off[:, :, k]) == sg)
            tail |= (mem & (np.cumsum(mem, 1) <= k_side))[:, 64:].any(1)
    return int(tail.sum())


@pytest.mark.parametrize("select", [lp.SELECT_NEAREST, lp.SELECT_OCTANT])
def test_neighbor_lists_k_max_80(select):
    """k_max = 80 (the jet's 20-80 neighbours): lists of up to 64 prefilter hits
    come from the tile kernel, longer ones from the per-particle kernel; both
    bit-exact."""
    st = inputs.jet_snapshot_3d(30_000)
    n = st["V"].shape[0]
    cfg = lp.make_config(3, n, radius_mode=lp.RADIUS_VOLUME, kappa=2.2, k_max=80, select=select)
    ocfg = _oracle_cfg(cfg)
    _, ocnt, otot, _ = oracle.neighbors(ocfg, st["x"], st["V"], st["m"], st["id"])
    assert (ocnt > 64).sum() > 100 and (otot > 80).sum() > 100 and ocnt.max() == 80
    ctx = lp.Context(cfg)
    ps = lp.ParticleSet.from_state(st)
    ctx.build_neighbors(ps)
    torch.cuda.synchronize()
    _check_lists(ctx, ps, st, ocfg)
    assert ctx.stats()["n_overflow"] == (otot > 80).sum()
    ctx.close()


@pytest.mark.parametrize("select", [lp.SELECT_NEAREST, lp.SELECT_OCTANT])
@pytest.mark.parametrize("prec,tol", [(lp.PREC_FP32, 1e-5), (lp.PREC_FP64, 1e-12)])
def test_step_jet_snapshot_k_max_80(prec, tol, select):
    """One step of the jet snapshot with k_max = 80: some one-sided stencils
    take members past list position 63 (found by the fits' tail scan)."""
    st = inputs.jet_snapshot_3d(30_000)
    n = st["V"].shape[0]
    cfg = lp.make_config(3, n, precision=prec, kappa=2.2, k_max=80, gamma=inputs.JET_GAMMA,
                         s_ref=inputs.field_scales(st), limiter=lp.LIM_FLAGGED, select=select)
    ocfg = _oracle_cfg(cfg)
    oidx, ocnt, _, _ = oracle.neighbors(ocfg, st["x"], st["V"], st["m"], st["id"])
    assert _stencil_tail_count(st, oidx, ocnt, cfg.k_side) > 20
    _step_parity(st, cfg, 0.0, tol, cfl=0.4)


def _octant_case(name):
    """States and configurations with octant-balanced selection where many lists
    are truncated: a dense cloud with a small capacity, the jet snapshot (the
    ambient particles next to the jet reach hundreds of jet particles), a
    periodic 2D shear layer with a small capacity, and an exact lattice (many
    equal distances, so the (d2, id) tie rule decides ranks)."""
    if name == "3d-cloud-k24":
        st = inputs.gas_cloud_3d(12_000, seed=9)
        return st, lp.make_config(3, 12_000, kappa=3.0, k_max=24, select=lp.SELECT_OCTANT)
    if name == "3d-jet-snapshot":
        st = inputs.jet_snapshot_3d(30_000)
        return st, lp.make_config(3, st["V"].shape[0], kappa=2.2, k_max=64, select=lp.SELECT_OCTANT)
    if name == "2d-periodic-kh-k16":
        st = inputs.kh_2d(7_001, 0.03, seed=5)
        return st, lp.make_config(2, st["V"].shape[0], kappa=2.2, k_max=16, periodic=(1, 1, 0),
                                  box_lo=(0, 0, 0), box_hi=(1, 1, 1), select=lp.SELECT_OCTANT)
    n = 21 ** 3
    # an unjittered lattice: shells of equal distance
    g = np.stack(np.meshgrid(*[np.arange(21) / 21.0] * 3, indexing="ij"), 0).reshape(3, -1)
    st = {"x": [g[0].copy(), g[1].copy(), g[2].copy()], "V": np.ones(n), "u": [np.zeros(n)] * 3,
          "P": np.ones(n), "m": np.ones(n), "id": np.arange(n, dtype=np.uint32), "n_fluid": n}
    return st, lp.make_config(3, n, radius_mode=lp.RADIUS_FIXED, radius=2.2 / 21, k_max=20,
                              select=lp.SELECT_OCTANT)


@pytest.mark.parametrize("sched", [0, lp.SCHED_QUERY_WARP])
@pytest.mark.parametrize("name", ["3d-cloud-k24", "3d-jet-snapshot", "2d-periodic-kh-k16", "3d-exact-lattice-k20"])
def test_octant_selection_lists_bit_exact(name, sched):
    """Octant-balanced selection (Sec. 2.2 step 4): the lists equal the oracle's,
    bit for bit, whether the tile kernel hands the truncated particles to the
    per-particle kernel or that kernel runs every particle."""
    st, cfg = _octant_case(name)
    ctx = lp.Context(cfg)
    ctx.set_schedule(sched)
    ps = lp.ParticleSet.from_state(st)
    ctx.build_neighbors(ps)
    torch.cuda.synchronize()
    _check_lists(ctx, ps, st, _oracle_cfg(cfg))
    s = ctx.stats()
    assert s["n_overflow"] > 0, s
    ctx.close()


def test_octant_selection_agrees_with_nearest_within_capacity():
    """With at most k_max inside the radius the two selections give the same
    list; where they differ, the octant-balanced list covers more octants."""
    st = inputs.jet_snapshot_3d(30_000)
    n = st["V"].shape[0]
    out = {}
    for sel in (lp.SELECT_NEAREST, lp.SELECT_OCTANT):
        cfg = lp.make_config(3, n, kappa=2.2, k_max=64, select=sel)
        ctx = lp.Context(cfg)
        ps = lp.ParticleSet.from_state(st)
        ctx.build_neighbors(ps)
        ids, lists, tot, d2, _ = gpu_neighbor_ids(ctx, ps)
        out[sel] = {int(p): (list(l), int(t), float(d)) for p, l, t, d in zip(ids, lists, tot, d2)}
        ctx.close()
    x = np.stack(st["x"], 1)
    more = 0
    for pid, (ln, tn, dn) in out[lp.SELECT_NEAREST].items():
        lo, to, do = out[lp.SELECT_OCTANT][pid]
        assert tn == to and dn == do
        if tn <= 64:
            assert ln == lo
        else:
            octs = lambda l: len({tuple((x[j] - x[pid]) >= 0.0) for j in l})
            assert octs(lo) >= octs(ln)
            more += octs(lo) > octs(ln)
    assert more > 0


@pytest.mark.parametrize("prec,tol", [(lp.PREC_FP32, 1e-5), (lp.PREC_FP64, 1e-12)])
def test_step_jet_snapshot_octant_selection(prec, tol):
    """One CFL step of the jet snapshot with octant-balanced lists: the ambient
    particles next to the jet fit stencils that reach the ambient side too."""
    st = inputs.jet_snapshot_3d(30_000)
    n = st["V"].shape[0]
    cfg = lp.make_config(3, n, precision=prec, kappa=2.2, k_max=64, gamma=inputs.JET_GAMMA,
                         s_ref=inputs.field_scales(st), limiter=lp.LIM_FLAGGED, select=lp.SELECT_OCTANT)
    errs, stats, ndiff = _step_parity(st, cfg, 0.0, tol, cfl=0.4)
    assert stats["n_overflow"] > 0, stats


def test_octant_coverage_check():
    """The all-octant coverage check of the central stencils
    (lp_octant_coverage): the particles whose list misses one of the 8 sign
    patterns of the offsets (exactly 0 counted as positive) are the ones the
    CPU finds on the oracle's lists (the cloud's edge particles, whose lists
    have no outward members)."""
    st = inputs.gas_cloud_3d(20_037, seed=4)
    n = st["V"].shape[0]
    cfg = lp.make_config(3, n, kappa=2.2, k_max=64)
    ctx = lp.Context(cfg)
    ps = lp.ParticleSet.from_state(st)
    ctx.build_neighbors(ps)
    gap = torch.zeros(n, dtype=torch.uint8, device="cuda")
    ngap = ctx.octant_coverage(gap)
    ids = ps.id.cpu().numpy().astype(np.int64)
    g = by_id(ids, gap.cpu().numpy())
    ctx.close()
    oidx, ocnt, _, _ = oracle.neighbors(_oracle_cfg(cfg), st["x"], st["V"], st["m"], st["id"])
    x = np.stack(st["x"], 1)
    want = np.array([len(set(map(tuple, (x[oidx[i, :ocnt[i]]] - x[i]) >= 0.0))) < 8 for i in range(n)])
    print("octant gaps: %d of %d" % (ngap, n))
    assert ngap == int(want.sum()) > 0
    assert np.array_equal(g.astype(bool), want)


def test_neighbor_lists_scattered_tiles():
    """Two far-apart clusters and a sprinkle of isolated points: tiles of 32
    consecutive particles that straddle them span too many cells and are left
    to the per-particle kernel; every list is still the oracle's."""
    rng = np.random.default_rng(12)
    a = rng.uniform(0.0, 0.05, size=(3, 1000))
    b = rng.uniform(0.0, 0.05, size=(3, 1013)) + 0.9
    c = rng.uniform(0.0, 1.0, size=(3, 45))
    x = np.concatenate([a, b, c], axis=1)
    n = x.shape[1]
    st = {"x": [x[0].copy(), x[1].copy(), x[2].copy()], "V": np.ones(n), "u": [np.zeros(n)] * 3, "P": np.ones(n),
          "m": np.ones(n), "id": np.arange(n, dtype=np.uint32), "n_fluid": n}
    cfg = lp.make_config(3, n, radius_mode=lp.RADIUS_FIXED, radius=0.012, k_max=64)
    ctx = lp.Context(cfg)
    ps = lp.ParticleSet.from_state(st)
    ctx.build_neighbors(ps)
    torch.cuda.synchronize()
    _check_lists(ctx, ps, st, _oracle_cfg(cfg))
    s = ctx.stats()
    assert 0 < s["n_query_fallback"] < n
    ctx.close()


def test_neighbor_empty_and_single():
    cfg = lp.make_config(3, 16, radius_mode=lp.RADIUS_FIXED, radius=0.1, k_max=8)
    ctx = lp.Context(cfg)
    st = inputs.uniform_box_3d(2, 0.5)
    st = inputs.take(st, np.arange(1))
    ps = lp.ParticleSet.from_state(st)
    ctx.build_neighbors(ps)
    cnt, tot, idx, d2, keys = ctx.export_neighbors(1)
    assert int(cnt[0]) == 0 and np.isinf(d2.cpu().numpy()[0])
    st0 = inputs.take(st, np.arange(0))
    ps0 = lp.ParticleSet.from_state(st0)
    ctx.build_neighbors(ps0)      # n = 0 is a no-op
    ctx.close()


def test_capacity_and_state_errors():
    cfg = lp.make_config(3, 10, radius_mode=lp.RADIUS_FIXED, radius=0.1, k_max=8)
    ctx = lp.Context(cfg)
    st = inputs.uniform_box_3d(3, 0.2)       # 27 particles > capacity 10
    ps = lp.ParticleSet.from_state(st)
    with pytest.raises(lp.LPError) as e:
        ctx.build_neighbors(ps)
    assert e.value.code == lp.ERR_CAPACITY
    with pytest.raises(lp.LPError) as e:
        ctx.gfd_derivs(ps, [ps.P])
    assert e.value.code in (lp.ERR_STATE, lp.ERR_ARG)
    ctx.close()


# ---------------------------------------------------------------------------
# GFD derivatives (config-2 shape at reduced size)
# ---------------------------------------------------------------------------

def _deriv_case(prec, noise, nf, n_side=22, refine=lp.REFINE_AUTO):
    h = 1.0 / n_side
    x, fields, coeffs = inputs.gfd_lattice_workload(n_side, h, noise, nfields=nf)
    n = x[0].shape[0]
    st = {"x": x, "V": np.ones(n), "u": [np.zeros(n)] * 3, "P": np.ones(n), "m": np.ones(n),
          "id": np.arange(n, dtype=np.uint32), "n_fluid": n}
    cfg = lp.make_config(3, n, precision=prec, radius_mode=lp.RADIUS_FIXED, radius=2.2 * h, k_max=64,
                         refine=refine)
    ctx = lp.Context(cfg)
    ps = lp.ParticleSet.from_state(st)
    ctx.build_neighbors(ps)
    ids = ps.id.cpu().numpy().astype(np.int64)
    dev_fields = [torch.as_tensor(f[ids], device="cuda") for f in fields]
    out = ctx.gfd_derivs(ps, dev_fields, lp.OUT_F64).cpu().numpy()
    ocfg = _oracle_cfg(cfg)
    oidx, ocnt, _, _ = oracle.neighbors(ocfg, x, st["V"], st["m"], st["id"])
    od, ost = oracle.gfd_central(ocfg, x, fields, ocnt, oidx)
    gd = np.stack([np.stack([by_id(ids, out[f][:, u]) for u in range(9)], axis=1) for f in range(nf)])
    ctx.close()
    return gd, od, coeffs, x


# Derivative tolerances.  Two backward-stable least-squares solvers (Givens on
# the GPU, pivoted Householder in the oracle) agree to ~cond(A) * m * n * u per
# solution component: cond ~ 30 after column scaling, m n ~ 400, so ~1.3e-12 in
# FP64 (u = 1.1e-16); bound 1e-11.  In FP32 the gradient is bounded by
# ~cond * 3u ~ 1e-5; the second derivatives carry only the b_H = H S^2 / 2 part
# of b = g S + H S^2 / 2, so their error is amplified by |g| S / |b_H| ~ 20-40 on
# this workload: ~cond * u * 40 ~ 1e-4; bound 1e-3.
FP64_DERIV_TOL = 1e-11
FP32_GRAD_TOL = 1e-5
FP32_HESS_TOL = 1e-3


@pytest.mark.parametrize("nf", [1, 5])
def test_gfd_derivs_fp64_matches_oracle(nf):
    gd, od, _, _ = _deriv_case(lp.PREC_FP64, 1e-6, nf)
    for f in range(nf):
        for u in range(9):
            assert normwise(gd[f][:, u], od[f][:, u]) < FP64_DERIV_TOL, (f, u)


@pytest.mark.parametrize("nf", [1, 5])
def test_gfd_derivs_fp32_matches_oracle(nf):
    gd, od, _, _ = _deriv_case(lp.PREC_FP32, 1e-6, nf)
    for f in range(nf):
        e1 = max(normwise(gd[f][:, u], od[f][:, u]) for u in range(3))
        e2 = max(normwise(gd[f][:, u], od[f][:, u]) for u in range(3, 9))
        assert e1 < FP32_GRAD_TOL, (f, e1)
        assert e2 < FP32_HESS_TOL, (f, e2)


def test_refinement_step_buys_fp32_accuracy():
    """The correction pass of the central fit (on by default) is what brings the
    FP32 gradients inside the 1e-5 bound; without it (NEVER) the error of the
    normal equations (~cond^2 u) remains.  AUTO corrects only the stencils
    below the ratio; a well-conditioned stencil's first solution is already
    within about cond^2 u, so its correction may round to nothing and AUTO
    may equal ALWAYS."""
    errs = {}
    for mode in (lp.REFINE_ALWAYS, lp.REFINE_AUTO, lp.REFINE_NEVER):
        gd, od, _, _ = _deriv_case(lp.PREC_FP32, 1e-6, 1, refine=mode)
        errs[mode] = max(normwise(gd[0][:, u], od[0][:, u]) for u in range(3))
    assert errs[lp.REFINE_ALWAYS] < FP32_GRAD_TOL
    assert errs[lp.REFINE_ALWAYS] <= errs[lp.REFINE_AUTO] <= errs[lp.REFINE_NEVER] < 1e-2, errs
    assert errs[lp.REFINE_NEVER] > 10 * errs[lp.REFINE_ALWAYS], errs


def test_gfd_derivs_fp32_noise_free_vs_analytic():
    gd, od, coeffs, x = _deriv_case(lp.PREC_FP32, 0.0, 1)
    c, g, H = coeffs[0]
    X = np.stack(x)
    grad = (g[:, None] + H @ X).T
    assert normwise(gd[0][:, :3], grad) < FP32_GRAD_TOL
    hess = np.array([H[0, 0], H[1, 1], H[2, 2], H[0, 1], H[0, 2], H[1, 2]])
    assert np.abs(gd[0][:, 3:] - hess).max() / np.abs(hess).max() < FP32_HESS_TOL


def test_fits_on_a_drifted_lattice():
    """A perfect lattice moved by a tiny amount (offsets of ~1e-16 where the
    lattice had exact zeros): stencil rows that are almost zero in a column
    meet rows that are not.  The square-root-free rotations must not lose the
    column (no fallback to the linear fit, derivatives as the oracle's)."""
    n_side, h = 12, 1.0 / 12
    x = inputs.jittered_lattice_3d(n_side, h, 0.0, seed=1)        # the perfect lattice
    rng = np.random.default_rng(3)
    x = [a + h * 1e-15 * rng.standard_normal(a.shape[0]) for a in x]
    c, g0, H = inputs.random_quadratic_3d(2)
    fields = [inputs.quadratic_values(x, c, g0, H)]
    n = x[0].shape[0]
    st = {"x": x, "V": np.ones(n), "u": [np.zeros(n)] * 3, "P": np.ones(n), "m": np.ones(n),
          "id": np.arange(n, dtype=np.uint32), "n_fluid": n}
    for prec, tol in ((lp.PREC_FP64, FP64_DERIV_TOL), (lp.PREC_FP32, FP32_GRAD_TOL)):
        cfg = lp.make_config(3, n, precision=prec, radius_mode=lp.RADIUS_FIXED, radius=2.2 * h, k_max=64)
        ctx = lp.Context(cfg)
        ps = lp.ParticleSet.from_state(st)
        ctx.build_neighbors(ps)
        ids = ps.id.cpu().numpy().astype(np.int64)
        status = torch.zeros(n, dtype=torch.int32, device="cuda")
        out = ctx.gfd_derivs(ps, [torch.as_tensor(fields[0][ids], device="cuda")], lp.OUT_F64, status=status)
        stt = status.cpu().numpy()
        assert np.all((stt & 3) == 0), (prec, np.bincount(stt))      # no linear fallback, no failed fit
        ocfg = _oracle_cfg(cfg)
        oidx, ocnt, _, _ = oracle.neighbors(ocfg, x, st["V"], st["m"], st["id"])
        od, _ = oracle.gfd_central(ocfg, x, fields, ocnt, oidx)
        g = np.stack([by_id(ids, out.cpu().numpy()[0][:, u]) for u in range(9)], axis=1)
        for u in range(3):
            assert normwise(g[:, u], od[0][:, u]) < tol, (prec, u)
        ctx.close()


def test_onesided_derivs_match_oracle():
    st = inputs.smooth_wave_3d(14, 1.0 / 14)
    n = st["V"].shape[0]
    for prec, tol in ((lp.PREC_FP64, 1e-12), (lp.PREC_FP32, 2e-5)):
        cfg = lp.make_config(3, n, precision=prec, radius_mode=lp.RADIUS_VOLUME, kappa=2.2, k_max=64, k_side=8)
        ctx = lp.Context(cfg)
        ps = lp.ParticleSet.from_state(st)
        ctx.build_neighbors(ps)
        ids = ps.id.cpu().numpy().astype(np.int64)
        fields = [ps.V, ps.u[0], ps.u[1], ps.u[2], ps.P]
        out = ctx.onesided_derivs(ps, fields).cpu().numpy()
        ocfg = _oracle_cfg(cfg)
        oidx, ocnt, _, _ = oracle.neighbors(ocfg, st["x"], st["V"], st["m"], st["id"])
        of = [st["V"], st["u"][0], st["u"][1], st["u"][2], st["P"]]
        oo = oracle.gfd_onesided(ocfg, st["x"], of, ocnt, oidx)
        g = np.empty_like(out)
        g[ids] = out
        for f in range(5):
            e = normwise(g[..., f], oo[..., f])
            assert e < tol, (prec, f, e)
        ctx.close()


# ---------------------------------------------------------------------------
# one LP step
# ---------------------------------------------------------------------------

# Rate tolerances.  The state after a step, s + dt rate, hides rate errors
# behind the size of s, so the rates (s^{n+1} - s^n) / dt are compared too.
# Each rate is a sum of products of state values and derivatives (LW: s_t from
# first derivatives, dt/2 s_tt from products of first derivatives and from
# second derivatives; UW: one-sided first derivatives).  FP64: the derivatives
# agree to FP64_DERIV_TOL = 1e-11; a product of two such factors and the sums
# over axes stay within 1e-9.  FP32: where a rate is led by first derivatives
# (the velocity rates, -V grad P, and every rate of a moving state) its error is
# that of the gradients, FP32_GRAD_TOL, times at most 2 for a product and 3 for
# the sum over axes: 6e-5.  The V and P rates of a state at rest have no
# first-order term (div u = 0) and are led by the Laplacian of P; on these
# smooth workloads its FP32 error is cond(A) u ~ 30 x 6e-8 times the share of
# the curvature in b = g.d + d^T H d / 2, at most ~40 at the cloud's edge
# (|grad P| r / |H| h), i.e. 7e-5.  Bar: 1e-4 for every field.
RATE_TOL = {lp.PREC_FP64: {"V": 1e-9, "u": 1e-9, "P": 1e-9},
            lp.PREC_FP32: {"V": 1e-4, "u": 1e-4, "P": 1e-4}}


def _step_parity(st, cfg, dt, tol, cfl=0.4, check_dt=False):
    n = st["V"].shape[0]
    nf = cfg.dim + 2
    ctx = lp.Context(cfg)
    ps = lp.ParticleSet.from_state(st)
    flag = torch.empty(n, dtype=torch.uint8, device="cuda")
    phi = torch.empty((n, nf), dtype=torch.float32, device="cuda")
    rr = torch.empty((n, nf), dtype=torch.float32, device="cuda")
    ctx.step(ps, dt=dt, cfl=cfl, flag=flag, phi=phi, r=rr)
    torch.cuda.synchronize()
    stats = ctx.stats()
    ids = ps.id.cpu().numpy().astype(np.int64)
    ocfg = _oracle_cfg(cfg, st.get("n_fluid", 2**62))
    if dt <= 0:
        oidx, ocnt, _, od2 = oracle.neighbors(ocfg, st["x"], st["V"], st["m"], st["id"])
        odt = oracle.cfl_dt(ocfg, st["V"], st["P"], st["id"], od2, cfl)
        assert abs(stats["dt"] - odt) <= 1e-14 * odt
        dt_used = stats["dt"]
    else:
        dt_used = dt
    q = np.arange(n)
    o = oracle.step(ocfg, st, dt_used, query=q)
    gphi = by_id(ids, phi.cpu().numpy())
    gflag = by_id(ids, flag.cpu().numpy())
    # particles whose discrete decision differs must lie in the ambiguity band;
    # the oracle is re-run with the GPU's phi for them
    o, ndiff = parity.resolve(ocfg, st, q, cfg.precision, gflag, gphi, o, dt_used, max(3, n // 500))
    g = state_by_id(ps, st.get("n_fluid"))
    errs, rates = parity.field_and_rate_errors(cfg.dim, st, g, o, dt_used)
    print("ambiguous %d; field errors %s; rate errors %s" % (ndiff, errs, rates))
    ctx.close()
    for k, e in errs.items():
        assert e < tol, (k, e, errs)
    for k, e in rates.items():
        assert e < RATE_TOL[cfg.precision][k[0]], (k, e, rates)
    assert np.array_equal(g["m"], st["m"])
    return errs, stats, ndiff


def test_step_fp64_smooth_3d():
    st = inputs.smooth_wave_3d(14, 1.0 / 14)
    n = st["V"].shape[0]
    cfg = lp.make_config(3, n, precision=lp.PREC_FP64, kappa=2.2, k_max=64, gamma=1.4,
                         s_ref=inputs.field_scales(st), limiter=lp.LIM_PAPER)
    _step_parity(st, cfg, 2e-3, 1e-12)


def test_step_fp32_smooth_3d():
    st = inputs.smooth_wave_3d(14, 1.0 / 14)
    n = st["V"].shape[0]
    cfg = lp.make_config(3, n, precision=lp.PREC_FP32, kappa=2.2, k_max=64, gamma=1.4,
                         s_ref=inputs.field_scales(st), limiter=lp.LIM_FLAGGED)
    _step_parity(st, cfg, 2e-3, 1e-5)


@pytest.mark.parametrize("prec,tol", [(lp.PREC_FP32, 1e-5), (lp.PREC_FP64, 1e-12)])
def test_step_gas_cloud_cfl(prec, tol):
    st = inputs.gas_cloud_3d(20_037, seed=4)
    cfg = lp.make_config(3, 20_037, precision=prec, kappa=2.2, k_max=64, gamma=5.0 / 3.0,
                         s_ref=inputs.field_scales(st), limiter=lp.LIM_FLAGGED)
    _step_parity(st, cfg, 0.0, tol, cfl=0.4)


@pytest.mark.parametrize("prec,tol", [(lp.PREC_FP32, 1e-5), (lp.PREC_FP64, 1e-12)])
def test_step_jet_snapshot_cfl(prec, tol):
    """The jet-shaped snapshot: a 1e3 density jump with 10-64 neighbours per
    particle, truncated lists around the jet, ill-conditioned one-sided and
    central stencils at the interface (FP64 redo in the FP32 path)."""
    st = inputs.jet_snapshot_3d(30_000)
    n = st["V"].shape[0]
    cfg = lp.make_config(3, n, precision=prec, kappa=2.2, k_max=64, gamma=inputs.JET_GAMMA,
                         s_ref=inputs.field_scales(st), limiter=lp.LIM_FLAGGED)
    errs, stats, ndiff = _step_parity(st, cfg, 0.0, tol, cfl=0.4)
    assert stats["n_overflow"] > 0 and stats["n_flagged"] > 0, stats


def test_step_sod_fp64_and_frozen_ghosts():
    st = inputs.sod_1d(889, 111)
    n = st["V"].shape[0]
    cfg = lp.make_config(1, n, precision=lp.PREC_FP64, radius_mode=lp.RADIUS_KSIDE, k_max=8, k_per_side=4,
                         k_side=1, gamma=1.4, s_ref=inputs.field_scales(st), n_fluid=st["n_fluid"])
    _step_parity(st, cfg, 0.0, 1e-12, cfl=0.4)


def test_step_kh_periodic_2d():
    st = inputs.kh_2d(6_000, 0.03, seed=5)
    n = st["V"].shape[0]
    for prec, tol in ((lp.PREC_FP64, 1e-12), (lp.PREC_FP32, 1e-5)):
        cfg = lp.make_config(2, n, precision=prec, kappa=2.2, k_max=40, gamma=1.4, periodic=(1, 1, 0),
                             box_lo=(0, 0, 0), box_hi=(1, 1, 1), s_ref=inputs.field_scales(st))
        _step_parity(st, cfg, 1e-3, tol)


def test_uniform_state_exact_on_gpu():
    st = inputs.uniform_box_3d(12, 1.0 / 12, vel=(0.3, -0.2, 0.1))
    n = st["V"].shape[0]
    cfg = lp.make_config(3, n, precision=lp.PREC_FP32, kappa=2.2, k_max=64, s_ref=inputs.field_scales(st))
    ctx = lp.Context(cfg)
    ps = lp.ParticleSet.from_state(st)
    ctx.step(ps, dt=0.01)
    g = state_by_id(ps, n)
    assert np.array_equal(g["V"], st["V"]) and np.array_equal(g["P"], st["P"])
    for k in range(3):
        assert np.array_equal(g["u"][k], st["u"][k])
        assert np.array_equal(g["x"][k], st["x"][k] + 0.01 * st["u"][k])
    ctx.close()


def test_multi_step_sod_fp64_tracks_oracle():
    st = inputs.sod_1d(222, 28)
    n = st["V"].shape[0]
    cfg = lp.make_config(1, n, precision=lp.PREC_FP64, radius_mode=lp.RADIUS_KSIDE, k_max=8, k_per_side=4,
                         k_side=1, gamma=1.4, s_ref=inputs.field_scales(st), n_fluid=st["n_fluid"])
    ocfg = _oracle_cfg(cfg, st["n_fluid"])
    ctx = lp.Context(cfg)
    ps = lp.ParticleSet.from_state(st)
    ost = dict(st)
    for _ in range(25):
        ctx.step(ps, dt=0.0, cfl=0.4)
        dt = ctx.stats()["dt"]
        o = oracle.step(ocfg, ost, dt)
        ost = dict(ost, x=o["x"], V=o["V"], u=o["u"], P=o["P"])
    g = state_by_id(ps, st["n_fluid"])
    assert normwise(g["P"], ost["P"]) < 1e-10
    assert normwise(g["u"][0], ost["u"][0]) < 1e-10
    ctx.close()


def test_last_step_ends_at_t_end():
    """With t_end set, the CFL step is clipped so that the last step lands on
    t_end exactly, and a simulation already there does not move."""
    st = inputs.gas_cloud_3d(5_000, seed=4)
    n = st["V"].shape[0]
    base = lp.make_config(3, n, kappa=2.2, k_max=64, gamma=5.0 / 3.0, s_ref=inputs.field_scales(st))
    ctx = lp.Context(base)
    ps = lp.ParticleSet.from_state(st)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.step(ps, dt=0.0, cfl=0.4, t=t)
    dt0 = ctx.stats()["dt"]
    ctx.close()
    t_end = 1.5 * dt0
    cfg = lp.make_config(3, n, kappa=2.2, k_max=64, gamma=5.0 / 3.0, s_ref=inputs.field_scales(st), t_end=t_end)
    ctx = lp.Context(cfg)
    ps = lp.ParticleSet.from_state(st)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.step(ps, dt=0.0, cfl=0.4, t=t)
    assert ctx.stats()["dt"] == dt0 and float(t.cpu()[0]) == dt0
    ctx.step(ps, dt=0.0, cfl=0.4, t=t)
    assert float(t.cpu()[0]) == t_end
    before = ps.to_state(n)
    ctx.step(ps, dt=0.0, cfl=0.4, t=t)
    after = ps.to_state(n)
    assert float(t.cpu()[0]) == t_end and ctx.stats()["dt"] == 0.0
    assert ctx.stats()["status"] == 0
    o = np.argsort(before["id"]); p = np.argsort(after["id"])
    for f in ("V", "P"):
        assert np.array_equal(before[f][o], after[f][p])
    for k in range(3):
        assert np.array_equal(before["x"][k][o], after["x"][k][p])
    ctx.close()
