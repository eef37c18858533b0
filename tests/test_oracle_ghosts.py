"""Pins of the oracle's free-surface ghost particles (Sec. 2.2 step 3: where a
particle's neighbourhood is incomplete in an axis direction, ghost particles
complete it).  Reading: direction (k, side) is incomplete when fewer than
min_per_side list members lie strictly on that side along axis k; the ghost
sits one nearest-neighbour distance away along that axis, with the particle's
mass, specific volume and velocity, the ghost pressure, and the id
ghost_base + 2 dim id + 2k + side.  The lattice cases are worked by hand."""
import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _square(n_side=5, h=0.1):
    g = np.stack(np.meshgrid(np.arange(n_side) * h, np.arange(n_side) * h, indexing="ij"), 0).reshape(2, -1)
    n = g.shape[1]
    return {"x": [g[0].copy(), g[1].copy()], "V": np.full(n, 2.0), "u": [np.full(n, 0.5), np.full(n, -0.25)],
            "P": np.ones(n), "m": np.full(n, 3.0), "id": np.arange(n, dtype=np.uint32)}


def _cfg(h=0.1, k_max=64):
    return oracle.make_config(2, radius_mode=oracle.RADIUS_FIXED, radius=1.5 * h, k_max=k_max)


def test_square_lattice_edges_and_corners():
    st = _square()
    g = oracle.free_surface_ghosts(_cfg(), st, min_per_side=1, p_ghost=0.0, ghost_base=1000)
    ids = list(g["id"])
    # particle (a, b) has id 5 a + b and x = (0.1 a, 0.1 b); its directions are
    # 0: -x, 1: +x, 2: -y, 3: +y.  Corners have two empty directions, edge
    # particles one, the nine interior particles none: 4 * 2 + 12 = 20 ghosts
    assert len(ids) == 20
    want = []
    for a in range(5):
        for b in range(5):
            pid = 5 * a + b
            dirs = [d for d, empty in enumerate([a == 0, a == 4, b == 0, b == 4]) if empty]
            want += [1000 + 4 * pid + d for d in dirs]
    assert ids == want
    # the ghost of corner (0, 0) in direction -x sits at (-0.1, 0): one
    # nearest-neighbour distance (0.1) away; state copied, pressure 0
    r = ids.index(1000 + 0)
    assert g["x"][0][r] == 0.0 - 0.1 and g["x"][1][r] == 0.0
    assert g["V"][r] == 2.0 and g["m"][r] == 3.0 and g["P"][r] == 0.0
    assert g["u"][0][r] == 0.5 and g["u"][1][r] == -0.25
    # the ghost of edge particle (4, 2) (id 22) in direction +x at (0.5, 0.2)
    r = ids.index(1000 + 4 * 22 + 1)
    assert g["x"][0][r] == 0.4 + 0.1 and g["x"][1][r] == 0.2


def test_min_per_side_counts_the_half_space():
    # radius 1.5 h: particle (1, 2) (id 7) has three members with x offset -h
    # ((0,1), (0,2), (0,3)) and none at -2h; (0, 2) has none on that side
    st = _square()
    g3 = oracle.free_surface_ghosts(_cfg(), st, min_per_side=3, p_ghost=0.0, ghost_base=1000)
    g4 = oracle.free_surface_ghosts(_cfg(), st, min_per_side=4, p_ghost=0.0, ghost_base=1000)
    assert 1000 + 4 * 7 + 0 not in set(g3["id"])
    assert 1000 + 4 * 7 + 0 in set(g4["id"])
    # edge particles in a corner's neighbourhood have two members on their
    # short side along the edge: (0, 1) (id 1) sees (0, 0) and (1, 0) at y - h
    assert 1000 + 4 * 1 + 2 in set(g3["id"])
    assert 1000 + 4 * 1 + 2 not in set(oracle.free_surface_ghosts(_cfg(), st, min_per_side=2, ghost_base=1000)["id"])


def test_pressure_frozen_and_isolated_particles():
    st = _square()
    # particles with id >= n_fluid get no ghosts; an isolated particle (no
    # neighbour) gets none either
    cfg = oracle.make_config(2, radius_mode=oracle.RADIUS_FIXED, radius=0.15, k_max=64, n_fluid=5)
    g = oracle.free_surface_ghosts(cfg, st, min_per_side=1, p_ghost=0.25, ghost_base=1000)
    assert all((int(i) - 1000) // 4 < 5 for i in g["id"])
    assert np.all(g["P"] == 0.25)
    lone = {"x": [np.array([0.0, 5.0]), np.array([0.0, 5.0])], "V": np.ones(2), "u": [np.zeros(2)] * 2,
            "P": np.ones(2), "m": np.ones(2), "id": np.arange(2, dtype=np.uint32)}
    assert oracle.free_surface_ghosts(_cfg(), lone, ghost_base=1000)["id"].size == 0


def test_ghosts_complete_the_neighbourhood():
    """After adding the ghosts, every fluid particle of the block has at least
    one list member on each side of each axis."""
    st = _square()
    g = oracle.free_surface_ghosts(_cfg(), st, min_per_side=1, ghost_base=1000)
    both = {k: (np.concatenate([st[k], g[k]]) if k != "x" and k != "u" else
                [np.concatenate([a, b]) for a, b in zip(st[k], g[k])]) for k in ("x", "V", "u", "P", "m", "id")}
    n = both["V"].shape[0]
    cfg = oracle.make_config(2, radius_mode=oracle.RADIUS_FIXED, radius=0.15, k_max=64, n_fluid=25)
    g2 = oracle.free_surface_ghosts(cfg, both, min_per_side=1, ghost_base=1000)
    assert g2["id"].size == 0
