"""Free-surface ghost particles on the GPU (lp_free_surface_ghosts,
lp_remove_ghosts) against the oracle (Sec. 2.2 step 3; the reading is in
lp.h): the ghosts' ids, positions (bit for bit) and states; one step with the
ghosts frozen in place; their removal."""
import numpy as np
import pytest

import oracle
from paper_2206_11998_gb300 import inputs, lp
from tests import parity
from tests.gpu_util import ensure_built

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GHOST_BASE = 2 ** 31


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    oracle.build()


def _by_id(st):
    o = np.argsort(st["id"], kind="stable")
    return {"x": [a[o] for a in st["x"]], "V": st["V"][o], "u": [a[o] for a in st["u"]], "P": st["P"][o],
            "m": st["m"][o], "id": st["id"][o]}


def _gpu_ghosts(st, cfg, min_per_side, p_ghost):
    n = st["V"].shape[0]
    dim = len(st["x"])
    ctx = lp.Context(cfg)
    ps = lp.ParticleSet.with_capacity(st, n * (1 + 2 * dim))
    added = ctx.free_surface_ghosts(ps, min_per_side=min_per_side, p_ghost=p_ghost, ghost_base=GHOST_BASE)
    torch.cuda.synchronize()
    all_ = ps.to_state()
    ctx.close()
    g = {k: ([a[n:] for a in v] if isinstance(v, list) else v[n:]) for k, v in all_.items()}
    f = {k: ([a[:n] for a in v] if isinstance(v, list) else v[:n]) for k, v in all_.items()}
    return added, g, f


def _same_ghosts(g, o):
    g, o = _by_id(g), _by_id(o)
    assert np.array_equal(g["id"], o["id"])
    for k in range(len(g["x"])):
        assert np.array_equal(g["x"][k], o["x"][k]), k
        assert np.array_equal(g["u"][k], o["u"][k]), k
    for f in ("V", "P", "m"):
        assert np.array_equal(g[f], o[f]), f


def test_square_lattice_ghosts_equal_the_oracle():
    h = 0.1
    gr = np.stack(np.meshgrid(np.arange(5) * h, np.arange(5) * h, indexing="ij"), 0).reshape(2, -1)
    n = gr.shape[1]
    st = {"x": [gr[0].copy(), gr[1].copy()], "V": np.full(n, 2.0), "u": [np.full(n, 0.5), np.full(n, -0.25)],
          "P": np.ones(n), "m": np.full(n, 3.0), "id": np.arange(n, dtype=np.uint32)}
    cfg = lp.make_config(2, n * 5, radius_mode=lp.RADIUS_FIXED, radius=1.5 * h, k_max=64, n_fluid=n)
    added, g, f = _gpu_ghosts(st, cfg, 1, 0.0)
    ocfg = oracle.make_config(2, radius_mode=oracle.RADIUS_FIXED, radius=1.5 * h, k_max=64, n_fluid=n)
    o = oracle.free_surface_ghosts(ocfg, st, 1, 0.0, GHOST_BASE)
    assert added == 20 == o["id"].size
    _same_ghosts(g, o)
    # the fluid particles are the input's, permuted into key order
    assert np.array_equal(np.sort(f["id"]), st["id"])


@pytest.mark.parametrize("min_per_side", [1, 3])
def test_cloud_ghosts_equal_the_oracle(min_per_side):
    st = inputs.gas_cloud_3d(20_037, seed=4)
    n = st["V"].shape[0]
    cfg = lp.make_config(3, n * 7, kappa=2.2, k_max=64, n_fluid=n)
    added, g, _ = _gpu_ghosts(st, cfg, min_per_side, 0.0)
    ocfg = oracle.make_config(3, kappa=2.2, k_max=64, n_fluid=n)
    o = oracle.free_surface_ghosts(ocfg, st, min_per_side, 0.0, GHOST_BASE)
    print("min_per_side %d: %d ghosts for %d particles" % (min_per_side, added, n))
    assert added == o["id"].size and added > 0
    _same_ghosts(g, o)


def test_capacity_is_checked_before_appending():
    st = inputs.gas_cloud_3d(5_000, seed=4)
    n = st["V"].shape[0]
    ctx = lp.Context(lp.make_config(3, n * 7, kappa=2.2, k_max=64, n_fluid=n))
    ps = lp.ParticleSet.with_capacity(st, n + 1)
    with pytest.raises(lp.LPError) as e:
        ctx.free_surface_ghosts(ps, min_per_side=2, ghost_base=GHOST_BASE)
    assert e.value.code == lp.ERR_CAPACITY and ps.n == n
    # ghosts must be frozen: a ghost base below n_fluid is refused
    ps = lp.ParticleSet.with_capacity(st, 7 * n)
    with pytest.raises(lp.LPError):
        ctx.free_surface_ghosts(ps, ghost_base=n - 1)
    ctx.close()


@pytest.mark.parametrize("prec,tol,rtol", [(lp.PREC_FP32, 1e-5, 1e-4), (lp.PREC_FP64, 1e-12, 1e-9)])
def test_step_with_ghosts_matches_the_oracle(prec, tol, rtol):
    """One CFL step of the cloud with its free-surface ghosts frozen in place
    (vacuum pressure), then the ghosts removed: the fluid state and rates equal
    the oracle's step of the same combined state (estimator decisions inside
    the ambiguity band are resolved as in the other step tests)."""
    st = inputs.gas_cloud_3d(20_037, seed=4)
    n = st["V"].shape[0]
    sref = inputs.field_scales(st)
    cfg = lp.make_config(3, n * 7, precision=prec, kappa=2.2, k_max=64, gamma=5.0 / 3.0, s_ref=sref,
                         limiter=lp.LIM_FLAGGED, n_fluid=n)
    ctx = lp.Context(cfg)
    ps = lp.ParticleSet.with_capacity(st, n * 7)
    added = ctx.free_surface_ghosts(ps, min_per_side=2, p_ghost=0.0, ghost_base=GHOST_BASE)
    both = _by_id(ps.to_state(n))          # fluid (ids 0..n-1) first, then the ghosts
    nt = ps.n
    flag = torch.empty(nt, dtype=torch.uint8, device="cuda")
    phi = torch.empty((nt, 5), dtype=torch.float32, device="cuda")
    ctx.step(ps, dt=0.0, cfl=0.4, flag=flag, phi=phi)
    torch.cuda.synchronize()
    dt = ctx.stats()["dt"]
    ids = ps.id[:nt].cpu().numpy().astype(np.uint32).astype(np.int64)
    fluid = ids < n
    gflag = np.empty(n, np.uint8)
    gphi = np.empty((n, 5), np.float32)
    gflag[ids[fluid]] = flag.cpu().numpy()[fluid]
    gphi[ids[fluid]] = phi.cpu().numpy()[fluid]
    removed = ctx.remove_ghosts(ps, GHOST_BASE)
    torch.cuda.synchronize()
    assert removed == added > 0 and ps.n == n
    g = _by_id(ps.to_state())
    assert np.array_equal(g["id"], np.arange(n, dtype=np.uint32))
    ocfg = oracle.make_config(3, gamma=5.0 / 3.0, kappa=2.2, k_max=64, s_ref=sref, limiter=oracle.LIM_FLAGGED,
                              n_fluid=n)
    q = np.arange(n)
    o = oracle.step(ocfg, both, dt, query=q)
    o, ndiff = parity.resolve(ocfg, both, q, prec, gflag, gphi, o, dt, max(3, n // 500))
    s0 = {"V": st["V"], "P": st["P"], "u": st["u"]}
    errs, rates = parity.field_and_rate_errors(3, s0, g, o, dt)
    print("ghosts %d; ambiguous %d; field errors %s; rate errors %s" % (added, ndiff, errs, rates))
    for k in ("V", "u0", "u1", "u2", "P"):
        assert errs[k] < tol, (k, errs)
        assert rates[k] < rtol, (k, rates)
    ctx.close()
