"""Pins of the oracle's exact Riemann solver and of the full LP scheme on the
Sod shock tube (ideal gas, gamma = 1.4).

* The exact solution satisfies, by substitution, the Rankine-Hugoniot jump
  conditions across the shock, the isentrope and Riemann invariant across the
  rarefaction, and pressure/velocity continuity across the contact; its star
  state matches the textbook values in tests/golden/sod_star_state.txt.
* The LP oracle run to t = 0.2 converges to it: the L1 errors of density,
  velocity and pressure decrease as the particle count doubles.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2206_11998_gb300 import inputs

G = 1.4
LEFT, RIGHT = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sod_star_state.txt")


def _golden():
    vals = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals


def test_star_state_matches_textbook(oracle_lib):
    gv = _golden()
    ps, us = oracle.riemann_star(G, LEFT, RIGHT)
    assert abs(ps - gv["p_star"]) < 1e-5 and abs(us - gv["u_star"]) < 1e-5
    t = 0.2
    xs = np.array([0.5 + 0.5 * us * t, 0.5 + 1.1 * us * t])   # either side of the contact
    r, u, p = oracle.riemann_exact(G, LEFT, RIGHT, 0.5, t, xs)
    assert abs(r[0] - gv["rho_star_left"]) < 1e-5 and abs(r[1] - gv["rho_star_right"]) < 1e-5


def test_jump_conditions_by_substitution(oracle_lib):
    t = 0.2
    ps, us = oracle.riemann_star(G, LEFT, RIGHT)
    xs = np.linspace(0.0, 1.0, 20001)
    r, u, p = oracle.riemann_exact(G, LEFT, RIGHT, 0.5, t, xs)
    # shock: the last point where the state differs from the right state
    js = np.nonzero(np.abs(r - RIGHT[0]) > 1e-12)[0][-1]
    S = (xs[js] - 0.5) / t
    r1, u1, p1 = r[js], u[js], p[js]
    r0, u0, p0 = RIGHT
    E = lambda rr, uu, pp: pp / (G - 1) + 0.5 * rr * uu * uu
    # mass, momentum, energy fluxes in the shock frame (S known to grid spacing)
    tol = 2e-3
    assert abs((r1 * (u1 - S)) - (r0 * (u0 - S))) < tol
    assert abs((r1 * u1 * (u1 - S) + p1) - (r0 * u0 * (u0 - S) + p0)) < tol
    assert abs(((E(r1, u1, p1) + p1) * u1 - S * E(r1, u1, p1)) - ((E(r0, u0, p0) + p0) * u0 - S * E(r0, u0, p0))) < tol
    # rarefaction: p / rho^gamma and u + 2c/(gamma-1) constant from the left state
    fan = (r < 1 - 1e-9) & (xs < 0.5)
    c = np.sqrt(G * p / r)
    assert np.abs(p[fan] / r[fan] ** G - 1.0).max() < 1e-12
    assert np.abs(u[fan] + 2 * c[fan] / (G - 1) - 2 * np.sqrt(G) / (G - 1)).max() < 1e-12
    # contact: p and u continuous, density jumps
    k = np.argmin(np.abs(xs - (0.5 + us * t)))
    assert abs(p[k - 2] - p[k + 2]) < 1e-12 and abs(u[k - 2] - u[k + 2]) < 1e-12
    assert abs(r[k - 2] - r[k + 2]) > 0.1


def run_sod(n_left, n_right, limiter=oracle.LIM_FLAGGED, t_end=0.2, cfl=0.4):
    st = inputs.sod_1d(n_left, n_right)
    cfg = oracle.make_config(1, gamma=G, radius_mode=oracle.RADIUS_KSIDE, k_max=8, k_per_side=4,
                             k_side=1, limiter=limiter, s_ref=inputs.field_scales(st),
                             n_fluid=st["n_fluid"])
    t = 0.0
    while t < t_end * (1 - 1e-12):
        idx, cnt, tot, d2 = oracle.neighbors(cfg, st["x"], st["V"], st["m"], st["id"])
        dt = min(oracle.cfl_dt(cfg, st["V"], st["P"], st["id"], d2, cfl), t_end - t)
        assert dt > 1e-9
        o = oracle.step(cfg, st, dt)
        st = dict(st, x=o["x"], V=o["V"], u=o["u"], P=o["P"])
        t += dt
    f = st["id"] < st["n_fluid"]
    r, u, p = oracle.riemann_exact(G, LEFT, RIGHT, 0.5, t, st["x"][0][f])
    return (np.mean(np.abs(1 / st["V"][f] - r)), np.mean(np.abs(st["u"][0][f] - u)),
            np.mean(np.abs(st["P"][f] - p)))


def test_sod_converges_to_exact_solution(oracle_lib):
    e1 = run_sod(222, 28)
    e2 = run_sod(444, 56)
    for a, b in zip(e1, e2):
        assert b < 0.85 * a
    assert e2[0] < 0.02 and e2[1] < 0.03 and e2[2] < 0.012


def test_sod_upwind_only_is_first_order_and_stable(oracle_lib):
    e = run_sod(444, 56, limiter=oracle.LIM_UW)
    assert e[0] < 0.03 and e[2] < 0.02
