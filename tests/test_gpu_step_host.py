"""lp_step_host: one step on host-resident particles.

The host entry point copies the state in (part of it on a second stream while
the keys sort) and, for page-locked arrays, lets the kernels write the new
state straight into host memory.  It must leave in the host arrays exactly
what lp_step leaves in device arrays, bit for bit, with page-locked and with
ordinary (pageable) host memory.
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


N = 50_000


def _cfg(st, **kw):
    return lp.make_config(3, N, kappa=2.2, k_max=64, gamma=5.0 / 3.0, s_ref=inputs.field_scales(st), **kw)


def _host_state(ps):
    return {"x": [a.numpy().copy() for a in ps.x], "V": ps.V.numpy().copy(), "u": [a.numpy().copy() for a in ps.u],
            "P": ps.P.numpy().copy(), "m": ps.m.numpy().copy(), "id": ps.id.numpy().astype(np.uint32)}


def _same(a, b):
    assert np.array_equal(a["id"], b["id"])
    for f in ("V", "P", "m"):
        assert np.array_equal(a[f], b[f]), f
    for d in range(3):
        assert np.array_equal(a["x"][d], b["x"][d]), d
        assert np.array_equal(a["u"][d], b["u"][d]), d


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("sched", [lp.SCHED_FUSED, lp.SCHED_SPLIT])
def test_host_step_equals_device_step(pinned, sched):
    st = inputs.gas_cloud_3d(N, seed=31)
    stream = torch.cuda.Stream()
    # device reference
    c1 = lp.Context(_cfg(st))
    c1.set_schedule(sched)
    ps = lp.ParticleSet.from_state(st)
    flag1 = torch.empty(N, dtype=torch.uint8, device="cuda")
    phi1 = torch.empty((N, 5), dtype=torch.float32, device="cuda")
    for _ in range(2):
        c1.step(ps, dt=0.0, cfl=0.4, flag=flag1, phi=phi1, stream=stream)
    stream.synchronize()
    ref = ps.to_state()
    s1 = c1.stats(stream=stream)
    c1.close()
    # host arrays
    c2 = lp.Context(_cfg(st))
    c2.set_schedule(sched)
    hs = lp.ParticleSet.from_state_host(st, pinned=pinned)
    assert hs.V.is_pinned() == pinned
    flag2 = torch.empty(N, dtype=torch.uint8, device="cuda")
    phi2 = torch.empty((N, 5), dtype=torch.float32, device="cuda")
    for _ in range(2):
        c2.step_host(hs, dt=0.0, cfl=0.4, flag=flag2, phi=phi2, stream=stream)
    stream.synchronize()
    got = _host_state(hs)
    s2 = c2.stats(stream=stream)
    c2.close()
    _same(ref, got)
    assert torch.equal(flag1, flag2)
    assert torch.equal(phi1, phi2)
    for k in ("n_flagged", "n_fp64_redo", "n_nonfinite", "steps", "dt"):
        assert s1[k] == s2[k], k


@pytest.mark.parametrize("prec", [lp.PREC_FP32, lp.PREC_FP64])
def test_host_step_periodic_2d(prec):
    """The 2D periodic shear layer (minimum-image offsets, positions wrapped by
    the mover) through the host path, both precisions."""
    st = inputs.kh_2d(8_000, 0.03, seed=7)
    n = st["V"].shape[0]
    cfg = lp.make_config(2, n, precision=prec, kappa=2.2, k_max=40, gamma=1.4, periodic=(1, 1, 0),
                         box_lo=(0, 0, 0), box_hi=(1, 1, 1), s_ref=inputs.field_scales(st))
    c1 = lp.Context(cfg)
    ps = lp.ParticleSet.from_state(st)
    for _ in range(3):
        c1.step(ps, dt=0.0, cfl=0.4)
    torch.cuda.synchronize()
    c2 = lp.Context(cfg)
    hs = lp.ParticleSet.from_state_host(st)
    for _ in range(3):
        c2.step_host(hs, dt=0.0, cfl=0.4)
    torch.cuda.synchronize()
    a, b = ps.to_state(), _host_state(hs)
    assert np.array_equal(a["id"], b["id"])
    for f in ("V", "P", "m"):
        assert np.array_equal(a[f], b[f]), f
    for d in range(2):
        assert np.array_equal(a["x"][d], b["x"][d]) and np.array_equal(a["u"][d], b["u"][d]), d
    c1.close()
    c2.close()


def test_host_step_fixed_dt_and_time():
    st = inputs.gas_cloud_3d(N, seed=32)
    c1 = lp.Context(_cfg(st))
    ps = lp.ParticleSet.from_state(st)
    t1 = torch.zeros(1, dtype=torch.float64, device="cuda")
    c1.step(ps, dt=1e-4, t=t1)
    torch.cuda.synchronize()
    c2 = lp.Context(_cfg(st))
    hs = lp.ParticleSet.from_state_host(st)
    t2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    c2.step_host(hs, dt=1e-4, t=t2)
    torch.cuda.synchronize()
    _same(ps.to_state(), _host_state(hs))
    assert float(t1.item()) == float(t2.item()) == 1e-4
    c1.close()
    c2.close()


def test_host_step_errors_and_empty():
    st = inputs.gas_cloud_3d(N, seed=33)
    batched = lp.Context(_cfg(st, max_sims=4))
    hs = lp.ParticleSet.from_state_host(st)
    with pytest.raises(lp.LPError) as e:
        batched.step_host(hs, dt=1e-4)
    assert e.value.code == lp.ERR_STATE
    batched.close()
    small = lp.Context(lp.make_config(3, 100, kappa=2.2, k_max=64))
    with pytest.raises(lp.LPError) as e:
        small.step_host(hs, dt=1e-4)               # more particles than the capacity
    assert e.value.code == lp.ERR_CAPACITY
    empty = {"x": [np.zeros(0)] * 3, "V": np.zeros(0), "u": [np.zeros(0)] * 3, "P": np.zeros(0), "m": np.zeros(0),
             "id": np.zeros(0, dtype=np.uint32)}
    small.step_host(lp.ParticleSet.from_state_host(empty, pinned=False), dt=1e-4)
    torch.cuda.synchronize()
    small.close()
