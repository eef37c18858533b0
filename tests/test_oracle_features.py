"""Pins of the oracle's learned-estimator inputs, CFL step and update safeguard
(CPU only).

The eight inputs are recomputed here from their definitions with an
independent least-squares solver (numpy's lstsq on the same Taylor rows) and a
brute-force neighbour set; the CFL step from its definition with a brute-force
nearest distance; the safeguard from its stated behaviour (an inadmissible
update keeps the old state and sets the status bit).
"""
import numpy as np

import oracle
from paper_2206_11998_gb300 import inputs

GAMMA = 1.4
R = 0.23


def _state(seed=3):
    x = inputs.jittered_lattice_3d(7, 0.1, 0.2, seed=seed)
    X, Y, Z = x
    n = X.shape[0]
    # smooth positive fields with cubic parts: the second-order fit is not exact,
    # so the residual input is non-trivial
    P = 2.0 + 0.3 * X - 0.2 * Y + 0.1 * Z + 0.4 * X * X - 0.3 * Y * Z + 0.5 * X ** 3 - 0.2 * Y ** 2 * Z
    V = 1.0 + 0.2 * Y + 0.1 * X * Z + 0.05 * Z ** 3
    u = [0.1 * X + 0.05 * Y * Y, -0.2 * Y + 0.1 * X * Z, 0.3 * Z + 0.02 * X ** 3]
    st = {"x": [a.copy() for a in x], "V": V, "u": u, "P": P, "m": np.full(n, 1e-3),
          "id": np.arange(n, dtype=np.uint32), "n_fluid": n}
    return st


def _brute(st, i):
    X = np.stack(st["x"])
    d = X - X[:, i:i + 1]
    d2 = (d * d).sum(axis=0)
    js = np.nonzero((d2 <= R * R) & (np.arange(d2.size) != i))[0]
    return js, d[:, js], d2[js]


def _fit(d, b):
    rows = np.stack([d[0], d[1], d[2], 0.5 * d[0] ** 2, 0.5 * d[1] ** 2, 0.5 * d[2] ** 2,
                     d[0] * d[1], d[0] * d[2], d[1] * d[2]], axis=1)
    sol, *_ = np.linalg.lstsq(rows, b, rcond=None)
    res = b - rows @ sol
    return sol, res


def _t(f):
    return np.log1p(10.0 * abs(f))


def _curv(sol, ell):
    g = np.abs(sol[:3])
    h = np.abs(sol[3:6])
    best = 0.0
    for k in range(3):
        if g[k] < 0.5 * g.max():
            continue
        den = g[k] + ell * h[k]
        best = max(best, ell * h[k] / den if den > 0 else 0.0)
    return best


def test_features_match_definition(oracle_lib):
    st = _state()
    n = st["V"].shape[0]
    cfg = oracle.make_config(3, gamma=GAMMA, radius_mode=oracle.RADIUS_FIXED, radius=R, k_max=64)
    q = np.arange(0, n, 7)
    got = oracle.features(cfg, st, query=q)
    for r, i in enumerate(q):
        js, d, d2 = _brute(st, i)
        assert 9 <= js.size <= 64
        ell = np.sqrt(d2.min())
        Pi, Vi = st["P"][i], st["V"][i]
        bP = st["P"][js] - Pi
        sP, resP = _fit(d, bP)
        sV, _ = _fit(d, st["V"][js] - Vi)
        div = sum(_fit(d, st["u"][k][js] - st["u"][k][i])[0][k] for k in range(3))
        c = np.sqrt(GAMMA * Pi * Vi)
        want = np.array([
            _t(ell * np.linalg.norm(sP[:3]) / Pi),
            _t(ell * np.linalg.norm(sV[:3]) / Vi),
            _t(_curv(sP, ell)),
            _t(_curv(sV, ell)),
            np.sign(div) * _t(ell * div / c),
            _t(max(0.0, bP.max()) / Pi),
            _t(-min(0.0, bP.min()) / Pi),
            _t(np.sqrt((resP ** 2).sum() / (bP ** 2).sum())),
        ])
        assert np.allclose(got[r], want, rtol=1e-8, atol=1e-10), (i, got[r], want)
    # the residual input is really exercised
    assert got[:, 7].max() > 1e-3


def test_features_of_exact_quadratic_have_zero_residual(oracle_lib):
    st = _state()
    X, Y, Z = st["x"]
    st["P"] = 2.0 + 0.3 * X + 0.4 * X * X - 0.3 * Y * Z
    cfg = oracle.make_config(3, gamma=GAMMA, radius_mode=oracle.RADIUS_FIXED, radius=R, k_max=64)
    got = oracle.features(cfg, st, query=np.arange(0, 343, 11))
    assert np.abs(got[:, 7]).max() < 1e-9


def test_cfl_step_matches_definition(oracle_lib):
    st = inputs.gas_cloud_3d(800, seed=5)
    n = st["V"].shape[0]
    st["n_fluid"] = n - 40                      # the last 40 ids are frozen: ignored
    cfg = oracle.make_config(3, gamma=5.0 / 3.0, kappa=2.2, k_max=64, n_fluid=n - 40)
    _, _, _, d2 = oracle.neighbors(cfg, st["x"], st["V"], st["m"], st["id"])
    X = np.stack(st["x"])
    best = np.inf
    for i in range(n - 40):
        d = X - X[:, i:i + 1]
        dd = (d * d).sum(axis=0)
        dd[i] = np.inf
        w = st["m"][i] * st["V"][i]
        inside = dd ** 3 <= 2.2 ** 6 * w * w
        if not inside.any():
            continue
        best = min(best, np.sqrt(dd[inside].min()) / np.sqrt(5.0 / 3.0 * st["P"][i] * st["V"][i]))
    dt = oracle.cfl_dt(cfg, st["V"], st["P"], st["id"], d2, 0.4)
    assert abs(dt - 0.4 * best) <= 1e-14 * best


def test_inadmissible_update_keeps_state(oracle_lib):
    st = inputs.smooth_wave_3d(8, 1.0 / 8, amp=0.4)
    cfg = oracle.make_config(3, gamma=GAMMA, kappa=2.2, k_max=64)
    o = oracle.step(cfg, st, 5.0)             # far beyond any stable step
    bad = (o["status"] & 8) != 0
    assert bad.any() and not bad.all()
    assert np.array_equal(o["V"][bad], st["V"][bad])
    assert np.array_equal(o["P"][bad], st["P"][bad])
    for k in range(3):
        assert np.array_equal(o["u"][k][bad], st["u"][k][bad])
    # the mover still uses the (kept) velocity: x + dt u
    for k in range(3):
        assert np.allclose(o["x"][k][bad], st["x"][k][bad] + 5.0 * st["u"][k][bad], rtol=0, atol=1e-12)
    ok = ~bad
    assert np.all(o["V"][ok] > 0) and np.all(o["P"][ok] > 0)
