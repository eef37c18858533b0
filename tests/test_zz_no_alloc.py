"""The allocation-free keys-and-order entry point, lp_sort_keys_noalloc.

Callers that cannot allocate device memory when they need the Morton order (a
host application whose own pool owns all device memory, or a latency-critical
loop that cannot absorb cudaMalloc's implicit device synchronisation) use this
entry point; its scratch is a fixed array inside the library.  Its output must
equal what the allocating path computes: the keys and permutation that
lp_build_neighbors produces with a default configuration, bit for bit (integer
work), on two calls in a row (the second call reuses the array the first one
left behind).  Sizes above the fixed maximum are rejected.
"""
import numpy as np
import pytest

from paper_2206_11998_gb300 import inputs, lp
from tests.gpu_util import ensure_built

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()


def _reference(st):
    """Keys and permutation from the allocating path (lp_build_neighbors) with a
    default configuration of the state's dimension."""
    n = st["V"].shape[0]
    dim = len(st["x"])
    if dim == 1:
        cfg = lp.make_config(1, n, radius_mode=lp.RADIUS_KSIDE, k_max=8, k_per_side=4, k_side=1)
    else:
        cfg = lp.make_config(dim, n, radius_mode=lp.RADIUS_VOLUME, kappa=2.2, k_max=64 if dim == 3 else 40)
    ctx = lp.Context(cfg)
    ps = lp.ParticleSet.from_state(st)
    ctx.build_neighbors(ps)
    keys = ctx.export_neighbors(n)[4].cpu().numpy().view(np.uint64).copy()
    perm = ps.id.cpu().numpy().astype(np.int64)      # ids are the input indices
    ctx.close()
    return keys, perm


def _noalloc(st):
    n = st["V"].shape[0]
    x = [torch.as_tensor(a, device="cuda") for a in st["x"]]
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    lp.sort_keys_noalloc(x, keys, perm)
    torch.cuda.synchronize()
    return keys.cpu().numpy().view(np.uint64), perm.cpu().numpy().astype(np.int64)


def test_noalloc_matches_allocating_path_on_two_calls():
    a = inputs.gas_cloud_3d(120_001, seed=21)
    x = inputs.jittered_lattice_3d(64, 1.0 / 64, 0.2, seed=22)          # 262144 = the maximum
    n = x[0].shape[0]
    assert n == lp.NOALLOC_MAX_N
    b = {"x": x, "V": np.full(n, 1.0), "u": [np.zeros(n)] * 3, "P": np.ones(n), "m": np.full(n, 64.0 ** -3),
         "id": np.arange(n, dtype=np.uint32), "n_fluid": n}
    for st in (a, b):
        ref_keys, ref_perm = _reference(st)
        keys, perm = _noalloc(st)
        assert np.array_equal(perm, ref_perm)
        assert np.array_equal(keys, ref_keys)


def test_noalloc_rejects_sizes_above_the_maximum():
    n = lp.NOALLOC_MAX_N + 1
    x = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in range(3)]
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(lp.LPError) as e:
        lp.sort_keys_noalloc(x, keys, perm)
    assert e.value.code == lp.ERR_CAPACITY


def test_noalloc_1d_and_2d_on_two_calls():
    """1D: the keys are the order-preserving image of x and the sort runs over
    all 64 bits (eight passes); 2D: Morton keys sorted by their cell bits down
    to level 13.  Two calls in a row each, the second on the array the first
    left behind; ties (equal x in 1D) keep the input order."""
    rng = np.random.default_rng(31)
    n1 = 100_003
    x1 = rng.normal(0.0, 1.0, n1)
    x1[::7] = np.round(x1[::7], 2)                   # many exactly equal positions, negative and positive
    x1[5] = -0.0
    x1[6] = 0.0
    s1 = {"x": [x1], "V": np.full(n1, 1e-3), "u": [np.zeros(n1)], "P": np.ones(n1), "m": np.ones(n1),
          "id": np.arange(n1, dtype=np.uint32), "n_fluid": n1}
    s2 = inputs.kh_2d(150_000, 0.03, seed=32)
    s2 = dict(s2, x=[a - 0.3 for a in s2["x"]])      # not periodic here: a plain bounding cube
    for st in (s1, s2):
        ref_keys, ref_perm = _reference(st)
        for _ in range(2):
            keys, perm = _noalloc(st)
            assert np.array_equal(perm, ref_perm)
            assert np.array_equal(keys, ref_keys)
