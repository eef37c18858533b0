"""Pins of the oracle's time step (Sec. 2.1) against what the paper and the
mathematics fix, independently of the oracle's own formulas:

* Lax-Wendroff rates: s_t and s_tt recovered from two oracle steps are compared
  with the material derivatives of the Eulerian Euler equations evaluated by
  sympy (chain rule on explicit polynomial fields; no use of the commutation
  identity or of the derived multi-D formulas).
* Upwind rates: 1D values of the printed Eqs. eq_upwind_V/u/P with exact
  one-sided slopes; the 3D axis-sum reading reduces to them along every axis.
* The characteristic decomposition printed with Eq. euler6.
* Limiter values; uniform-state and Galilean invariance; frozen boundary
  particles; linear stability (LW keeps an acoustic wave, UW damps it).
"""
import numpy as np
import pytest

import oracle
from paper_2206_11998_gb300 import inputs

GAMMA = 1.4


def _lattice_state(n_side, h, seed, fields_fn):
    x = inputs.jittered_lattice_3d(n_side, h, 0.2, seed)
    n = x[0].shape[0]
    V, u, P = fields_fn(np.stack(x))
    return {"x": x, "V": V, "u": u, "P": P, "m": np.full(n, h ** 3) / V,
            "id": np.arange(n, dtype=np.uint32), "n_fluid": n}


def _rates_from_two_steps(cfg, st, i, dts):
    outs = [oracle.step(cfg, st, dt, query=[i]) for dt in dts]
    dim = cfg.dim
    s0 = np.array([st["V"][i]] + [st["u"][k][i] for k in range(dim)] + [st["P"][i]])
    r = []
    for o, dt in zip(outs, dts):
        s1 = np.array([o["V"][0]] + [o["u"][k][0] for k in range(dim)] + [o["P"][0]])
        r.append((s1 - s0) / dt)
    # (s1 - s0)/dt = s_t + dt/2 s_tt
    s_tt = (r[1] - r[0]) / (0.5 * (dts[1] - dts[0]))
    s_t = r[0] - 0.5 * dts[0] * s_tt
    return s_t, s_tt


def _sympy_rates(coef, pos, gamma):
    sp = pytest.importorskip("sympy")
    X = sp.symbols("x0:3")
    t = sp.Symbol("t")

    def quad(c):
        c0, g, H = c
        e = sp.Float(c0)
        for a in range(3):
            e += sp.Float(g[a]) * X[a]
            for b in range(3):
                e += sp.Rational(1, 2) * sp.Float(H[a][b]) * X[a] * X[b]
        return e

    V0 = quad(coef["V"]); P0 = quad(coef["P"]); U0 = [quad(c) for c in coef["u"]]
    grad = lambda f: [sp.diff(f, X[a]) for a in range(3)]
    div = lambda U: sum(sp.diff(U[a], X[a]) for a in range(3))
    adv = lambda U, f: sum(U[a] * sp.diff(f, X[a]) for a in range(3))
    # Eulerian rates of the Lagrangian Euler system (Sec. 2.1, Eqs. mass,
    # momentum, energy with e = P V / (gamma - 1)):
    EV = -adv(U0, V0) + V0 * div(U0)
    EU = [-adv(U0, U0[a]) - V0 * grad(P0)[a] for a in range(3)]
    EP = -adv(U0, P0) - gamma * P0 * div(U0)
    Vt_ = V0 + t * EV; Pt_ = P0 + t * EP; Ut_ = [U0[a] + t * EU[a] for a in range(3)]
    # material rates as functions of the (time-dependent) fields
    mat = [Vt_ * div(Ut_)] + [-Vt_ * grad(Pt_)[a] for a in range(3)] + [-gamma * Pt_ * div(Ut_)]
    sub = {X[a]: sp.Float(pos[a]) for a in range(3)}
    s_t, s_tt = [], []
    for R in mat:
        R0 = R.subs(t, 0)
        D = sp.diff(R, t).subs(t, 0) + adv(U0, R0)
        s_t.append(float(R0.subs(sub)))
        s_tt.append(float(D.subs(sub)))
    return np.array(s_t), np.array(s_tt)


def _rand_quad(rng, c0, scale):
    g = scale * rng.standard_normal(3)
    A = scale * rng.standard_normal((3, 3))
    return (c0, g, 0.5 * (A + A.T))


def _eval_quad(c, X):
    c0, g, H = c
    return c0 + g @ X + 0.5 * np.einsum("in,ij,jn->n", X, H, X)


def test_lax_wendroff_rates_match_material_derivatives_3d(oracle_lib):
    rng = np.random.default_rng(12)
    coef = {"V": _rand_quad(rng, 1.3, 0.3), "P": _rand_quad(rng, 2.0, 0.4),
            "u": [_rand_quad(rng, 0.2 * k, 0.5) for k in range(3)]}
    st = _lattice_state(9, 0.1, 5, lambda X: (_eval_quad(coef["V"], X),
                                              [_eval_quad(c, X) for c in coef["u"]],
                                              _eval_quad(coef["P"], X)))
    cfg = oracle.make_config(3, gamma=GAMMA, radius_mode=oracle.RADIUS_FIXED, radius=0.25,
                             k_max=64, limiter=oracle.LIM_LW)
    i = int(np.argmin(sum((a - 0.45) ** 2 for a in st["x"])))
    s_t, s_tt = _rates_from_two_steps(cfg, st, i, (0.01, 0.03))
    ref_t, ref_tt = _sympy_rates(coef, [a[i] for a in st["x"]], GAMMA)
    assert np.allclose(s_t, ref_t, rtol=1e-9, atol=1e-9 * np.abs(ref_t).max())
    assert np.allclose(s_tt, ref_tt, rtol=1e-6, atol=1e-6 * np.abs(ref_tt).max())


def test_lax_wendroff_1d_matches_printed_second_derivatives(oracle_lib):
    # Sec. 2.1: V_tt = -V V_x P_x - V^2 P_xx;  u_tt = g V u_x P_x + g V P u_xx;
    # P_tt = (g^2 + g) P u_x^2 + g V_x P P_x + g V P P_xx  (1D, all printed)
    st = inputs.sod_1d(60, 60, ghosts=4, right=(1.0, 0.0, 1.0))
    x = st["x"][0]
    cV, cu, cP = (0.9, 0.3, -0.7), (0.1, -0.4, 0.9), (1.5, 0.6, 0.5)
    q = lambda c: c[0] + c[1] * x + 0.5 * c[2] * x * x
    st["V"], st["u"], st["P"] = q(cV), [q(cu)], q(cP)
    cfg = oracle.make_config(1, gamma=GAMMA, radius_mode=oracle.RADIUS_KSIDE, k_max=8, k_per_side=4,
                             limiter=oracle.LIM_LW, n_fluid=st["n_fluid"])
    i = 40
    s_t, s_tt = _rates_from_two_steps(cfg, st, i, (0.01, 0.02))
    xi = x[i]
    V, u, P = q(cV)[i], q(cu)[i], q(cP)[i]
    Vx, ux, Px = cV[1] + cV[2] * xi, cu[1] + cu[2] * xi, cP[1] + cP[2] * xi
    Vxx, uxx, Pxx = cV[2], cu[2], cP[2]
    g = GAMMA
    ref_t = np.array([V * ux, -V * Px, -g * P * ux])
    ref_tt = np.array([-V * Vx * Px - V * V * Pxx,
                       g * V * ux * Px + g * V * P * uxx,
                       (g * g + g) * P * ux * ux + g * Vx * P * Px + g * V * P * Pxx])
    assert np.allclose(s_t, ref_t, rtol=1e-8, atol=1e-10)
    assert np.allclose(s_tt, ref_tt, rtol=1e-5, atol=1e-7)


def _uw_1d(V, P, ul, ur, Pl, Pr, g=GAMMA):
    # Eqs. eq_upwind_V, eq_upwind_u, eq_upwind_P with K = g P / V
    K = g * P / V
    sK = np.sqrt(K)
    return np.array([V / 2 * (ur + ul) - V / (2 * sK) * (Pr - Pl),
                     V * sK / 2 * (ur - ul) - V / 2 * (Pr + Pl),
                     -V * K / 2 * (ur + ul) + V * sK / 2 * (Pr - Pl)])


def _kinked(x, x0, c0, sl, sr):
    return c0 + np.where(x < x0, sl * (x - x0), sr * (x - x0))


def test_upwind_1d_matches_printed_equations(oracle_lib):
    st = inputs.sod_1d(50, 50, ghosts=4, right=(1.0, 0.0, 1.0))
    x = st["x"][0]
    i = 49
    x0 = x[i]   # kink at the particle: exact one-sided slopes
    st["V"] = _kinked(x, x0, 1.1, 0.2, -0.3)
    st["u"] = [_kinked(x, x0, 0.1, 0.7, -1.2)]
    st["P"] = _kinked(x, x0, 2.0, -0.5, 0.4)
    cfg = oracle.make_config(1, gamma=GAMMA, radius_mode=oracle.RADIUS_KSIDE, k_max=8, k_per_side=4,
                             k_side=1, limiter=oracle.LIM_UW, n_fluid=st["n_fluid"])
    dt = 1e-3
    o = oracle.step(cfg, st, dt, query=[i])
    got = (np.array([o["V"][0], o["u"][0][0], o["P"][0]]) - np.array([1.1, 0.1, 2.0])) / dt
    ref = _uw_1d(1.1, 2.0, 0.7, -1.2, -0.5, 0.4)
    assert np.allclose(got, ref, rtol=1e-10, atol=1e-12)


def _axis_state(axis, fV, fu, fP):
    h = 0.1
    g = (np.arange(9) + 0.5) * h
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    x = [X.ravel(), Y.ravel(), Z.ravel()]
    n = x[0].shape[0]
    i = int(np.argmin((x[0] - 0.45) ** 2 + (x[1] - 0.45) ** 2 + (x[2] - 0.45) ** 2))
    c = x[axis][i]
    u = [np.zeros(n) for _ in range(3)]
    u[axis] = fu(x[axis], c)
    st = {"x": x, "V": fV(x[axis], c), "u": u, "P": fP(x[axis], c), "m": np.full(n, h ** 3),
          "id": np.arange(n, dtype=np.uint32), "n_fluid": n}
    return st, i


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_upwind_3d_reduces_to_1d_along_each_axis(oracle_lib, axis):
    """The multi-D reading applies the 1D upwind operator along each axis with the
    normal velocity.  Fields varying along one axis only: (a) with a kink at the
    particle, the normal-velocity rate equals the printed 1D Eq. eq_upwind_u with
    the distinct left/right slopes; (b) with linear fields, the V and P rates
    equal Eqs. eq_upwind_V and eq_upwind_P (the other axes contribute nothing).
    """
    cfg = oracle.make_config(3, gamma=GAMMA, radius_mode=oracle.RADIUS_FIXED, radius=0.25, k_max=64,
                             k_side=8, limiter=oracle.LIM_UW)
    dt = 1e-3
    st, i = _axis_state(axis, lambda s, c: _kinked(s, c, 1.1, 0.2, -0.3),
                        lambda s, c: _kinked(s, c, 0.1, 0.7, -1.2),
                        lambda s, c: _kinked(s, c, 2.0, -0.5, 0.4))
    o = oracle.step(cfg, st, dt, query=[i])
    ref = _uw_1d(1.1, 2.0, 0.7, -1.2, -0.5, 0.4)
    assert abs((o["u"][axis][0] - 0.1) / dt - ref[1]) < 1e-9
    for k in range(3):
        if k != axis:   # left and right leaks of the kink cancel to round-off
            assert abs(o["u"][k][0]) < 1e-15
    st, i = _axis_state(axis, lambda s, c: 1.1 + 0.2 * (s - c), lambda s, c: 0.1 + 0.7 * (s - c),
                        lambda s, c: 2.0 - 0.5 * (s - c))
    o = oracle.step(cfg, st, dt, query=[i])
    got = np.array([(o["V"][0] - 1.1) / dt, (o["u"][axis][0] - 0.1) / dt, (o["P"][0] - 2.0) / dt])
    ref = _uw_1d(1.1, 2.0, 0.7, 0.7, -0.5, -0.5)
    assert np.allclose(got, ref, rtol=1e-9, atol=1e-11)


def test_characteristic_decomposition_printed_with_euler6():
    V, P = 0.8, 1.7
    K = GAMMA * P / V
    s = np.sqrt(K)
    A = V * np.array([[0, -1, 0], [0, 0, 1], [0, K, 0]])
    R = np.array([[1, 1, 1], [0, -s, s], [0, -K, -K]])
    Ri = np.array([[1, 0, 1 / K], [0, -1 / (2 * s), -1 / (2 * K)], [0, 1 / (2 * s), -1 / (2 * K)]])
    L = V * np.diag([0, s, -s])
    assert np.allclose(R @ Ri, np.eye(3))
    assert np.allclose(A @ R, R @ L)


def test_limiter_values(oracle_lib):
    assert oracle.phi(1.0) == 1.25
    assert oracle.phi(float("inf")) == 0.0
    assert abs(oracle.phi(1.5) - 1.25 * np.exp(1 - np.sqrt(1.5))) < 1e-15     # first branch at 3/2
    assert abs(oracle.phi(1.5 + 1e-12) - 1.25 * np.exp(-4.5 * (np.sqrt(1.5) - 1) ** 2)) < 1e-9
    assert 0.995 < oracle.phi(1.5) < 0.999 and 0.995 < oracle.phi(1.5 + 1e-9) < 0.997
    # r = (a/b + b/a)/2 >= 1 whenever a b > 0, and phi decreases on [1, inf)
    rs = np.linspace(1, 30, 300)
    ph = np.array([oracle.phi(r) for r in rs])
    assert np.all(np.diff(ph) < 0)


def test_uniform_state_is_preserved_exactly(oracle_lib):
    st = inputs.uniform_box_3d(7, 0.1, vel=(0.3, -0.2, 0.1))
    st["m"] = st["m"] * 1.0
    cfg = oracle.make_config(3, gamma=GAMMA, radius_mode=oracle.RADIUS_VOLUME, kappa=2.2, k_max=64,
                             limiter=oracle.LIM_PAPER, s_ref=inputs.field_scales(st))
    dt = 0.01
    o = oracle.step(cfg, st, dt)
    assert np.array_equal(o["V"], st["V"]) and np.array_equal(o["P"], st["P"])
    for k in range(3):
        assert np.array_equal(o["u"][k], st["u"][k])
        assert np.array_equal(o["x"][k], st["x"][k] + dt * st["u"][k])


def test_galilean_invariance(oracle_lib):
    st = inputs.smooth_wave_3d(9, 1.0 / 9)
    cfg = oracle.make_config(3, gamma=GAMMA, radius_mode=oracle.RADIUS_VOLUME, kappa=2.2, k_max=64,
                             limiter=oracle.LIM_FLAGGED, s_ref=inputs.field_scales(st))
    dt = 2e-3
    o1 = oracle.step(cfg, st, dt)
    c = np.array([0.37, -0.21, 0.05])
    st2 = dict(st, u=[st["u"][k] + c[k] for k in range(3)])
    o2 = oracle.step(cfg, st2, dt)
    assert np.allclose(o2["V"], o1["V"], rtol=1e-12, atol=0)
    assert np.allclose(o2["P"], o1["P"], rtol=1e-12, atol=0)
    for k in range(3):
        assert np.allclose(o2["u"][k] - c[k], o1["u"][k], rtol=0, atol=1e-12)
    assert np.array_equal(o1["flag"], o2["flag"])


def test_boundary_particles_frozen_and_mass_untouched(oracle_lib):
    st = inputs.sod_1d(40, 10, ghosts=4)
    cfg = oracle.make_config(1, gamma=GAMMA, radius_mode=oracle.RADIUS_KSIDE, k_max=8, k_per_side=4,
                             k_side=1, n_fluid=st["n_fluid"], s_ref=inputs.field_scales(st))
    o = oracle.step(cfg, st, 1e-3)
    g = st["id"] >= st["n_fluid"]
    assert np.array_equal(o["V"][g], st["V"][g]) and np.array_equal(o["x"][0][g], st["x"][0][g])
    assert not np.array_equal(o["V"][~g], st["V"][~g])


def _acoustic(lim, steps=150, N=100):
    x = (np.arange(N) + 0.5) / N
    amp = 1e-3
    s = np.sin(2 * np.pi * x)
    rho = 1 + amp * s
    st = {"x": [x], "V": 1 / rho, "u": [np.sqrt(GAMMA) * amp * s], "P": 1 + GAMMA * amp * s,
          "m": rho / N, "id": np.arange(N, dtype=np.uint32), "n_fluid": N}
    cfg = oracle.make_config(1, gamma=GAMMA, radius_mode=oracle.RADIUS_KSIDE, k_max=8, k_per_side=4,
                             k_side=1, limiter=lim, s_ref=(1, 1, 1), periodic=(1, 0, 0))
    for _ in range(steps):
        idx, cnt, tot, d2 = oracle.neighbors(cfg, st["x"], st["V"], st["m"], st["id"])
        dt = oracle.cfl_dt(cfg, st["V"], st["P"], st["id"], d2, 0.4)
        o = oracle.step(cfg, st, dt)
        st = dict(st, x=o["x"], V=o["V"], u=o["u"], P=o["P"])
    return np.abs(st["P"] - 1).max() / (GAMMA * amp)


def test_linear_stability_lw_keeps_uw_damps(oracle_lib):
    a_lw = _acoustic(oracle.LIM_LW)
    a_uw = _acoustic(oracle.LIM_UW)
    assert 0.98 < a_lw < 1.01
    assert a_uw < 0.97 and a_lw - a_uw > 0.03
