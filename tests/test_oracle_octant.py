"""Pins of the oracle's octant-balanced neighbour selection (Sec. 2.2 step 4:
the top members of a neighbour list must cover all directions, not just the
nearest).  Reading: when more than k_max particles lie inside the radius, the
k_max kept are taken round robin over the octants (quadrants in 2D), nearest
first in each, and stored in (d^2, id) order.  The cases below are small,
with the expected lists worked out by hand."""
import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _lists(pts, k_max, select, dim=2, periodic=(0, 0, 0), box=(0.0, 1.0), query=(0,)):
    pts = np.asarray(pts, dtype=np.float64)
    n = pts.shape[0]
    x = [pts[:, k].copy() for k in range(dim)]
    cfg = oracle.make_config(dim, radius_mode=oracle.RADIUS_FIXED, radius=100.0, k_max=k_max,
                             periodic=periodic, box_lo=(box[0],) * 3, box_hi=(box[1],) * 3, select=select)
    idx, cnt, tot, d2 = oracle.neighbors(cfg, x, np.ones(n), np.ones(n), np.arange(n, dtype=np.uint32),
                                         query=np.asarray(query, np.int64))
    return idx, cnt, tot, d2


# particle 0 at the origin; quadrant (x >= 0, y >= 0) holds the five nearest
# (distances 1..5), quadrant (x < 0, y >= 0) one at 10, quadrant (x < 0, y < 0)
# two at 11 and 12, quadrant (x >= 0, y < 0) none
CLUSTER = [(0.0, 0.0),
           (1.0, 0.0), (0.0, 2.0), (3.0, 0.0), (0.0, 4.0), (5.0, 0.0),   # indices 1..5
           (-10.0, 0.0),                                                  # 6
           (-11.0, -0.0001), (-12.0, -0.0001)]                            # 7, 8


def test_round_robin_over_quadrants():
    # ranks: quadrant 3 -> 1:0 2:1 3:2 4:3 5:4; quadrant 2 -> 6:0; quadrant 0 -> 7:0 8:1.
    # (rank, d2) order: 1, 6, 7 (rank 0), then 2, 8 (rank 1), ...; the first four,
    # in (d2, id) order, are 1, 2, 6, 7
    idx, cnt, tot, d2 = _lists(CLUSTER, 4, oracle.SELECT_OCTANT)
    assert cnt[0] == 4 and tot[0] == 8
    assert list(idx[0, :4]) == [1, 2, 6, 7]
    assert d2[0] == 1.0                     # the nearest distance is the nearest of all
    # the nearest-first selection keeps quadrant 3 only
    idx, cnt, tot, _ = _lists(CLUSTER, 4, oracle.SELECT_NEAREST)
    assert list(idx[0, :4]) == [1, 2, 3, 4]


def test_second_round_and_an_empty_quadrant():
    # k_max 6: rank 0 gives 1, 6, 7; rank 1 gives 2 and 8 (quadrant 2 has no
    # second member, quadrant 1 none at all); rank 2 gives 3
    idx, cnt, _, _ = _lists(CLUSTER, 6, oracle.SELECT_OCTANT)
    assert list(idx[0, :6]) == [1, 2, 3, 6, 7, 8]


def test_within_capacity_equals_nearest():
    a = _lists(CLUSTER, 8, oracle.SELECT_OCTANT)
    b = _lists(CLUSTER, 8, oracle.SELECT_NEAREST)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_zero_offset_counts_as_positive_side():
    # offsets exactly 0 along x go with x >= 0: 1 (0,-1) is in quadrant (x >= 0, y < 0),
    # 2 (0, 5) and 3 (0, 6) in (x >= 0, y >= 0), 4 (-7, 0) in (x < 0, y >= 0)
    pts = [(0.0, 0.0), (0.0, -1.0), (0.0, 5.0), (0.0, 6.0), (-7.0, 0.0)]
    idx, cnt, _, _ = _lists(pts, 3, oracle.SELECT_OCTANT)
    # rank 0: 1 (d 1), 2 (d 5), 4 (d 7); nearest-first would keep 1, 2, 3
    assert list(idx[0, :3]) == [1, 2, 4]


def test_periodic_axis_uses_the_minimum_image():
    # box [0, 1): seen from 0.05, the particle at 0.95 is 0.1 to the left (x < 0)
    pts = [(0.05, 0.5), (0.06, 0.5), (0.07, 0.5), (0.08, 0.5), (0.95, 0.5)]
    pts = np.asarray(pts)
    x = [pts[:, 0].copy(), pts[:, 1].copy()]
    cfg = oracle.make_config(2, radius_mode=oracle.RADIUS_FIXED, radius=0.2, k_max=2, periodic=(1, 1, 0),
                             box_lo=(0, 0, 0), box_hi=(1, 1, 1), select=oracle.SELECT_OCTANT)
    idx, cnt, tot, _ = oracle.neighbors(cfg, x, np.ones(5), np.ones(5), np.arange(5, dtype=np.uint32),
                                        query=np.array([0], np.int64))
    # quadrant (x >= 0, y >= 0): 1, 2, 3 (ranks 0, 1, 2); quadrant (x < 0, y >= 0): 4 (rank 0)
    assert tot[0] == 4
    assert list(idx[0, :2]) == [1, 4]


def test_3d_one_from_each_octant():
    # two particles in each of the 8 octants, the nearer at 1 + o/100, the
    # farther at 3 + o/100; k_max 8 keeps the nearer of each octant
    pts = [(0.0, 0.0, 0.0)]
    for o in range(8):
        s = np.array([1.0 if (o >> k) & 1 else -1.0 for k in range(3)]) / np.sqrt(3.0)
        pts.append(tuple(s * (1.0 + o / 100.0)))
        pts.append(tuple(s * (3.0 + o / 100.0)))
    idx, cnt, tot, _ = _lists(pts, 8, oracle.SELECT_OCTANT, dim=3)
    assert cnt[0] == 8 and tot[0] == 16
    assert list(idx[0, :8]) == [1 + 2 * o for o in range(8)]
    # nearest-first takes the same eight here: they are also the eight nearest
    idx2, _, _, _ = _lists(pts, 8, oracle.SELECT_NEAREST, dim=3)
    assert list(idx2[0, :8]) == list(idx[0, :8])
    # with k_max 4, rank 0 of octants 0..3 (the four nearest rank-0 members)
    idx, _, _, _ = _lists(pts, 4, oracle.SELECT_OCTANT, dim=3)
    assert list(idx[0, :4]) == [1, 3, 5, 7]


def test_selection_properties_on_a_random_cloud():
    """Properties that hold for any input: the kept members of each octant are
    a prefix of that octant's (d2, id) order; every non-empty octant keeps its
    nearest when k_max >= the number of non-empty octants; no octant keeps two
    more than another that still has members left out."""
    rng = np.random.default_rng(3)
    n = 400
    pts = rng.normal(size=(n, 3))
    x = [pts[:, k].copy() for k in range(3)]
    cfg = oracle.make_config(3, radius_mode=oracle.RADIUS_FIXED, radius=1.2, k_max=16,
                             select=oracle.SELECT_OCTANT)
    full = oracle.make_config(3, radius_mode=oracle.RADIUS_FIXED, radius=1.2, k_max=64)
    q = np.arange(0, n, 7, dtype=np.int64)
    ids = np.arange(n, dtype=np.uint32)
    idx, cnt, tot, _ = oracle.neighbors(cfg, x, np.ones(n), np.ones(n), ids, query=q)
    fidx, fcnt, ftot, _ = oracle.neighbors(full, x, np.ones(n), np.ones(n), ids, query=q)
    checked = 0
    for r, i in enumerate(q):
        if ftot[r] > 64 or ftot[r] <= 16:
            continue
        checked += 1
        allj = list(fidx[r, :fcnt[r]])                      # the in-radius set, (d2, id) order
        octs = {j: sum(1 << k for k in range(3) if pts[j, k] - pts[i, k] >= 0.0) for j in allj}
        kept = list(idx[r, :cnt[r]])
        assert cnt[r] == 16 and set(kept) <= set(allj)
        assert kept == [j for j in allj if j in set(kept)]     # stored in (d2, id) order
        per = {o: [j for j in allj if octs[j] == o] for o in range(8)}
        took = {o: [j for j in per[o] if j in set(kept)] for o in range(8)}
        for o in range(8):
            assert took[o] == per[o][:len(took[o])]            # a prefix of the octant's order
        short = [len(took[o]) for o in range(8) if len(took[o]) < len(per[o])]
        if short:
            assert max(len(took[o]) for o in range(8)) <= min(short) + 1
    assert checked > 10
