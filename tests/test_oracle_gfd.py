"""Pins of the oracle's GFD fits (Sec. 2.1, Eq. linear_system_axb).

A least-squares fit of a second-order Taylor polynomial reproduces any
quadratic exactly (the residual is zero), so the fitted first and second
derivatives must equal the analytic ones to round-off; a first-order fit
reproduces any linear field.  Any dropped term, wrong factor (e.g. the 1/2 on
the pure second derivatives) or transposed unknown fails these.
"""
import numpy as np
import pytest

import oracle
from paper_2206_11998_gb300 import inputs


def analytic_derivs_3d(g, H, X):
    # gradient g + H x, Hessian H, in the unknown order
    # (x, y, z, xx, yy, zz, xy, xz, yz)
    grad = g[:, None] + H @ X
    hess = np.array([H[0, 0], H[1, 1], H[2, 2], H[0, 1], H[0, 2], H[1, 2]])
    return np.concatenate([grad, np.repeat(hess[:, None], X.shape[1], axis=1)]).T


def test_central_fit_exact_on_quadratics_3d(oracle_lib):
    x, fields, coeffs = inputs.gfd_lattice_workload(n_side=10, h=0.1, noise=0.0, nfields=3)
    cfg = oracle.make_config(3, radius_mode=oracle.RADIUS_FIXED, radius=0.22, k_max=64)
    n = x[0].shape[0]
    ones = np.ones(n)
    idx, cnt, tot, d2 = oracle.neighbors(cfg, x, ones, ones, np.arange(n, dtype=np.uint32))
    der, st = oracle.gfd_central(cfg, x, fields, cnt, idx)
    assert np.all(st == 0)
    X = np.stack(x)
    for f, (c, g, H) in enumerate(coeffs):
        ref = analytic_derivs_3d(g, H, X)
        err = np.abs(der[f] - ref).max() / np.abs(ref).max()
        assert err < 1e-10, (f, err)


def test_central_fit_exact_on_quadratics_2d_paper_row(oracle_lib):
    # 2D row [h, k, h^2/2, k^2/2, hk] and unknowns (U_x, U_y, U_xx, U_yy, U_xy)
    rng = np.random.default_rng(3)
    n = 400
    x = [rng.uniform(0, 1, n), rng.uniform(0, 1, n)]
    a = rng.standard_normal(6)
    U = a[0] + a[1] * x[0] + a[2] * x[1] + 0.5 * a[3] * x[0] ** 2 + 0.5 * a[4] * x[1] ** 2 + a[5] * x[0] * x[1]
    cfg = oracle.make_config(2, radius_mode=oracle.RADIUS_FIXED, radius=0.15, k_max=64)
    ones = np.ones(n)
    idx, cnt, tot, d2 = oracle.neighbors(cfg, x, ones, ones, np.arange(n, dtype=np.uint32))
    der, st = oracle.gfd_central(cfg, x, [U], cnt, idx)
    ok = cnt >= 8
    ref = np.stack([a[1] + a[3] * x[0] + a[5] * x[1], a[2] + a[4] * x[1] + a[5] * x[0],
                    np.full(n, a[3]), np.full(n, a[4]), np.full(n, a[5])]).T
    assert np.abs(der[0][ok] - ref[ok]).max() < 1e-9


def test_central_fit_exact_1d(oracle_lib):
    st = inputs.sod_1d(30, 30, ghosts=4)
    x = st["x"][0]
    U = 0.3 - 2.0 * x + 1.7 * x * x
    cfg = oracle.make_config(1, radius_mode=oracle.RADIUS_KSIDE, k_max=8, k_per_side=4)
    idx, cnt, tot, d2 = oracle.neighbors(cfg, st["x"], st["V"], st["m"], st["id"])
    der, s = oracle.gfd_central(cfg, st["x"], [U], cnt, idx)
    assert np.abs(der[0][:, 0] - (-2.0 + 3.4 * x)).max() < 1e-9
    assert np.abs(der[0][:, 1] - 3.4).max() < 1e-6


def test_onesided_exact_on_linear_fields(oracle_lib):
    x = inputs.jittered_lattice_3d(8, 0.1, 0.2, seed=21)
    n = x[0].shape[0]
    g = np.array([0.7, -1.3, 2.1])
    U = 0.4 + g @ np.stack(x)
    cfg = oracle.make_config(3, radius_mode=oracle.RADIUS_FIXED, radius=0.22, k_max=64, k_side=8)
    ones = np.ones(n)
    idx, cnt, tot, d2 = oracle.neighbors(cfg, x, ones, ones, np.arange(n, dtype=np.uint32))
    os_ = oracle.gfd_onesided(cfg, x, [U], cnt, idx)
    for k in range(3):
        for s in range(2):
            assert np.abs(os_[:, k, s, 0] - g[k]).max() < 1e-10


def test_onesided_picks_the_side(oracle_lib):
    # kinked field |x - 0.5| * a: left/right derivatives differ at the kink
    st = inputs.sod_1d(50, 50, ghosts=4, right=(1.0, 0.0, 1.0))
    x = st["x"][0]
    U = np.where(x < 0.5, -1.5 * (x - 0.5), 2.5 * (x - 0.5))
    cfg = oracle.make_config(1, radius_mode=oracle.RADIUS_KSIDE, k_max=8, k_per_side=4, k_side=4)
    idx, cnt, tot, d2 = oracle.neighbors(cfg, st["x"], st["V"], st["m"], st["id"])
    os_ = oracle.gfd_onesided(cfg, st["x"], [U], cnt, idx)
    i = np.argmin(np.abs(x - 0.495))      # last particle left of the kink
    assert abs(os_[i, 0, 0, 0] + 1.5) < 1e-12
    j = np.argmin(np.abs(x - 0.505))      # first particle right of the kink
    assert abs(os_[j, 0, 1, 0] - 2.5) < 1e-12


def test_planar_stencil_falls_back_to_linear(oracle_lib):
    # all particles in the plane z = 0.5: the z columns vanish, the second-order
    # system is rank deficient and the first-order one too (dz column zero)
    rng = np.random.default_rng(4)
    n = 200
    x = [rng.uniform(0, 1, n), rng.uniform(0, 1, n), np.full(n, 0.5)]
    U = 1.0 + 2.0 * x[0] - x[1]
    cfg = oracle.make_config(3, radius_mode=oracle.RADIUS_FIXED, radius=0.3, k_max=64)
    ones = np.ones(n)
    idx, cnt, tot, d2 = oracle.neighbors(cfg, x, ones, ones, np.arange(n, dtype=np.uint32))
    der, st = oracle.gfd_central(cfg, x, [U], cnt, idx)
    assert np.all(st & oracle.ST_LINEAR_FALLBACK)
    assert np.all(st & oracle.ST_NO_FIT)
    assert np.all(der == 0.0)


def test_near_singular_second_order_falls_back(oracle_lib):
    # points on a line in 2D: second-order system rank deficient, first-order too
    n = 50
    t = np.linspace(0, 1, n)
    x = [t, 2 * t]
    cfg = oracle.make_config(2, radius_mode=oracle.RADIUS_FIXED, radius=0.2, k_max=64)
    ones = np.ones(n)
    idx, cnt, tot, d2 = oracle.neighbors(cfg, x, ones, ones, np.arange(n, dtype=np.uint32))
    der, st = oracle.gfd_central(cfg, x, [t], cnt, idx)
    assert np.all(st & oracle.ST_LINEAR_FALLBACK)
