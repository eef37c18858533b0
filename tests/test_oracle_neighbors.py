"""Pins of the oracle's neighbour search and Morton keys (CPU only).

The neighbour set of Sec. 2.2 steps 3-4 is {j != i : |x_j - x_i| <= R_i},
ordered by (d^2, id).  Each test recomputes it by brute force in numpy, an
implementation independent of the oracle's window search, and requires
bit-identical lists.
"""
import numpy as np
import pytest

import oracle
from paper_2206_11998_gb300 import inputs


def brute_lists(x, V, m, ids, mode, radius, kappa, k_max, periodic=(0, 0, 0), L=(1, 1, 1)):
    dim = len(x)
    n = x[0].shape[0]
    out = []
    for i in range(n):
        d = []
        for k in range(dim):
            dk = x[k] - x[k][i]
            if periodic[k]:
                h = 0.5 * L[k]
                dk = np.where(dk > h, dk - L[k], np.where(dk < -h, dk + L[k], dk))
            d.append(dk)
        d2 = d[0] * d[0]
        if dim > 1:
            d2 = d2 + d[1] * d[1]
        if dim > 2:
            d2 = d2 + d[2] * d[2]
        if mode == oracle.RADIUS_FIXED:
            ok = d2 <= radius * radius
        else:
            w = m[i] * V[i]
            k2 = kappa * kappa
            if dim == 3:
                ok = (d2 * d2) * d2 <= ((k2 * k2) * k2) * (w * w)
            elif dim == 2:
                ok = d2 * d2 <= (k2 * k2) * (w * w)
            else:
                ok = d2 <= k2 * (w * w)
        ok[i] = False
        js = np.nonzero(ok)[0]
        order = np.lexsort((ids[js], d2[js]))
        # the count before truncation saturates at 4 k_max
        out.append((js[order][:k_max], min(len(js), 4 * k_max), d2[js][order][0] if len(js) else np.inf))
    return out


def check(cfg, st, brute):
    idx, cnt, tot, d2 = oracle.neighbors(cfg, st["x"], st["V"], st["m"], st["id"])
    for i, (js, total, d2min) in enumerate(brute):
        assert cnt[i] == len(js)
        assert tot[i] == total
        assert np.array_equal(idx[i, :cnt[i]], js)
        assert d2[i] == d2min


def test_fixed_radius_3d_matches_brute_force(oracle_lib):
    x = inputs.jittered_lattice_3d(8, 0.1, 0.2, seed=11)
    n = x[0].shape[0]
    st = {"x": x, "V": np.ones(n), "m": np.ones(n), "id": np.arange(n, dtype=np.uint32)}
    cfg = oracle.make_config(3, radius_mode=oracle.RADIUS_FIXED, radius=0.22, k_max=64)
    check(cfg, st, brute_lists(x, st["V"], st["m"], st["id"], oracle.RADIUS_FIXED, 0.22, 0, 64))


def test_volume_radius_3d_with_truncation(oracle_lib):
    st = inputs.gas_cloud_3d(600, seed=3)
    # ids permuted so that id order differs from index order
    st["id"] = np.random.default_rng(0).permutation(600).astype(np.uint32)
    cfg = oracle.make_config(3, radius_mode=oracle.RADIUS_VOLUME, kappa=2.2, k_max=24)
    b = brute_lists(st["x"], st["V"], st["m"], st["id"], oracle.RADIUS_VOLUME, 0, 2.2, 24)
    assert max(t for _, t, _ in b) > 24        # truncation exercised
    assert max(t for _, t, _ in b) == 96       # and the saturated count
    check(cfg, st, b)


def test_volume_radius_jet_contrast(oracle_lib):
    """A 1e3 density jump: ambient radii ~10x the jet's, so ambient particles
    next to the jet see hundreds of jet particles (truncated to k_max, the
    count saturating at 4 k_max) while jet particles see few ambient ones."""
    st = inputs.jet_snapshot_3d(2500, l_jet=4.0, length=6.0, half_width=3.0)
    n = st["V"].shape[0]
    jet = st["V"] == 1.0
    assert 0 < (~jet).sum() < jet.sum()
    assert np.all(st["m"] == st["m"][0])            # equal masses
    cfg = oracle.make_config(3, radius_mode=oracle.RADIUS_VOLUME, kappa=2.2, k_max=32)
    b = brute_lists(st["x"], st["V"], st["m"], st["id"], oracle.RADIUS_VOLUME, 0, 2.2, 32)
    assert max(t for i, (_, t, _) in enumerate(b) if not jet[i]) == 128   # ambient lists saturate
    check(cfg, st, b)


def test_ties_broken_by_id_on_perfect_lattice(oracle_lib):
    g = (np.arange(6) + 0.5) * 0.25
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    x = [X.ravel(), Y.ravel(), Z.ravel()]
    n = x[0].shape[0]
    ids = np.random.default_rng(1).permutation(n).astype(np.uint32)
    st = {"x": x, "V": np.ones(n), "m": np.ones(n), "id": ids}
    # radius includes the 6 face and 12 edge neighbours (exact ties in d^2)
    cfg = oracle.make_config(3, radius_mode=oracle.RADIUS_FIXED, radius=0.36, k_max=10)
    b = brute_lists(x, st["V"], st["m"], ids, oracle.RADIUS_FIXED, 0.36, 0, 10)
    check(cfg, st, b)


def test_periodic_2d_minimum_image(oracle_lib):
    st = inputs.kh_2d(400, 0.03, seed=5)
    cfg = oracle.make_config(2, radius_mode=oracle.RADIUS_VOLUME, kappa=2.2, k_max=40,
                             periodic=(1, 1, 0), box_lo=(0, 0, 0), box_hi=(1, 1, 1))
    b = brute_lists(st["x"], st["V"], st["m"], st["id"], oracle.RADIUS_VOLUME, 0, 2.2, 40,
                    periodic=(1, 1, 0))
    check(cfg, st, b)
    # some list must cross the periodic boundary
    idx, cnt, _, _ = oracle.neighbors(cfg, st["x"], st["V"], st["m"], st["id"])
    x0 = st["x"][0]
    assert any(np.any(np.abs(x0[idx[i, :cnt[i]]] - x0[i]) > 0.5) for i in range(400))


def test_kside_1d(oracle_lib):
    st = inputs.sod_1d(40, 10, ghosts=4)
    cfg = oracle.make_config(1, radius_mode=oracle.RADIUS_KSIDE, k_max=8, k_per_side=4)
    idx, cnt, tot, d2 = oracle.neighbors(cfg, st["x"], st["V"], st["m"], st["id"])
    x = st["x"][0]
    for i in range(x.shape[0]):
        dx = x - x[i]
        left = np.nonzero(dx < 0)[0]
        right = np.nonzero(dx > 0)[0]
        left = left[np.lexsort((st["id"][left], dx[left] ** 2))][:4]
        right = right[np.lexsort((st["id"][right], dx[right] ** 2))][:4]
        both = np.concatenate([left, right])
        both = both[np.lexsort((st["id"][both], dx[both] ** 2))]
        assert np.array_equal(idx[i, :cnt[i]], both)


def test_morton_keys_by_hand(oracle_lib):
    # cube [0, 8) with 3 bits per axis: q = floor(x)
    pts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [3, 0, 0], [7, 7, 7], [5, 2, 6]], float)
    x = [pts[:, 0] + 0.5, pts[:, 1] + 0.5, pts[:, 2] + 0.5]
    keys = oracle.morton_keys(x, (0, 0, 0), 8.0, 3)
    # bit b of q_k lands at bit 3b + k
    def inter(q):
        return sum(((int(q[k]) >> b) & 1) << (3 * b + k) for b in range(3) for k in range(3))
    assert list(keys) == [inter(p) for p in pts.astype(int)]
    assert list(keys[:5]) == [0, 1, 2, 4, 9]
    assert keys[5] == 511


def test_morton_clamps_and_orders_2d(oracle_lib):
    x = [np.array([-1.0, 0.0, 0.999, 5.0]), np.array([0.0, 0.5, 0.999, 5.0])]
    keys = oracle.morton_keys(x, (0, 0), 1.0, 4)
    assert keys[0] == 0
    assert keys[3] == (1 << 8) - 1            # clamped to the last cell
    assert keys[2] == (1 << 8) - 1
    assert keys[1] == 0b10000000              # q = (0, 8): top bit of axis 1
