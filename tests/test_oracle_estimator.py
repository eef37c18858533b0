"""Pins of the oracle's state estimator and of the FLAGGED limiter rule
(Sec. 2.1: the ratio r of the one-sided derivatives, the limiter phi(r) and
the blend of Lax-Wendroff and upwind rates where the estimator flags).

The paper prints r for one field in 1D.  The readings for several axes and
fields are: an axis whose larger one-sided magnitude is below active_frac of
the largest over the axes is ignored; r is the maximum over the others; a
field whose one-sided derivatives are all below the flatness floor
(max|d| ell <= flat_eps max(|s|, s_ref)) has r = 1; a particle is flagged when
any field has r > 3/2, and then every field takes phi(r_s); unflagged
particles take phi = 1 (pure Lax-Wendroff).

Every expected value below is worked out by hand from those rules (the
arithmetic is written next to each case), so a dropped axis, a min in place
of the max, a reversed activity test, a per-field flag or a wrong flatness
scale fails one of them.
"""
import numpy as np
import pytest

import oracle


def r_of(sl, sr, ell=1.0, s_i=1.0, s_ref=0.0, flat_eps=1e-6, active_frac=0.5):
    return oracle.estimator_r(sl, sr, ell, s_i, s_ref, flat_eps, active_frac)


def test_one_axis_printed_ratio(oracle_lib):
    # r = (s_r / s_l + s_l / s_r) / 2
    assert r_of([2.0], [2.0]) == 1.0                       # equal slopes: smooth
    assert r_of([1.0], [2.0]) == 1.25                      # (2 + 1/2) / 2
    assert r_of([1.0], [4.0]) == 2.125                     # (4 + 1/4) / 2
    assert r_of([-1.0], [-2.0]) == 1.25                    # same sign, both negative
    assert r_of([2.0], [1.0]) == 1.25                      # symmetric in the two sides


def test_sign_change_gives_infinity(oracle_lib):
    assert np.isinf(r_of([1.0], [-0.5]))                   # an extremum between the sides
    assert np.isinf(r_of([0.0], [1.0]))                    # s_l s_r = 0 counts as a sign change
    assert oracle.phi(np.inf) == 0.0                       # and takes pure upwind


def test_inactive_axis_is_ignored(oracle_lib):
    # axis 0: slopes 1, 2 (G = 2, r_0 = 1.25); axis 1 changes sign but its
    # larger magnitude 0.1 is below 0.5 G = 1: ignored, r = 1.25
    assert r_of([1.0, 0.1], [2.0, -0.1]) == 1.25
    # the same sign change at magnitude 1.2 >= 1: active, r = inf
    assert np.isinf(r_of([1.0, 1.2], [2.0, -1.2]))


def test_activity_threshold_edges(oracle_lib):
    # G = 2 from axis 0; axis 1 slopes (0.25, g): r_1 = (g/0.25 + 0.25/g)/2
    # g = 0.99 < 0.5 G = 1: ignored, r = r_0 = 1.25
    assert r_of([1.0, 0.25], [2.0, 0.99]) == 1.25
    # g = 1.0 is not below 0.5 G: active, r = max(1.25, (4 + 1/4)/2) = 2.125
    assert r_of([1.0, 0.25], [2.0, 1.0]) == 2.125
    # a lower active_frac admits the 0.99 axis: r_1 = (3.96 + 0.25/0.99)/2
    r = r_of([1.0, 0.25], [2.0, 0.99], active_frac=0.1)
    assert abs(r - 0.5 * (3.96 + 0.25 / 0.99)) < 1e-15


def test_maximum_over_active_axes(oracle_lib):
    # r_0 = (2 + 1/2)/2 = 1.25, r_1 = (4 + 1/4)/2 = 2.125, r_2 = 1: the largest
    assert r_of([1.0, 1.0, 3.0], [2.0, 4.0, 3.0]) == 2.125
    # the order of the axes does not matter
    assert r_of([1.0, 3.0, 1.0], [4.0, 3.0, 2.0]) == 2.125


def test_flatness_floor(oracle_lib):
    # G = 3e-7; G ell = 3e-7 <= 1e-6 * max(|s_i| = 1, 0): locally constant, r = 1
    assert r_of([1e-7], [3e-7], ell=1.0, s_i=1.0) == 1.0
    # the same slopes over ell = 10: 3e-6 > 1e-6, r = (3 + 1/3)/2 = 5/3
    assert abs(r_of([1e-7], [3e-7], ell=10.0, s_i=1.0) - 5.0 / 3.0) < 1e-15
    # the scale is max(|s_i|, s_ref): |s_i| = 0.01 alone makes 3e-7 > 1e-8 ...
    assert abs(r_of([1e-7], [3e-7], ell=1.0, s_i=-0.01) - 5.0 / 3.0) < 1e-15
    # ... and s_ref = 1 raises the floor to 1e-6 again
    assert r_of([1e-7], [3e-7], ell=1.0, s_i=-0.01, s_ref=1.0) == 1.0
    # a field at rest (all one-sided derivatives zero) is flat, not a sign change
    assert r_of([0.0, 0.0, 0.0], [0.0, 0.0, 0.0], s_i=0.0) == 1.0
    # a floor test on the largest axis, not on each: G = 2 is not flat, and the
    # tiny axis is inactive
    assert r_of([1.0, 1e-9], [2.0, -1e-9]) == 1.25


def test_r_is_at_least_one_and_scale_free(oracle_lib):
    rng = np.random.default_rng(0)
    for _ in range(2000):
        d = int(rng.integers(1, 4))
        sl = rng.normal(size=d) * 10.0 ** rng.uniform(-3, 3)
        sr = rng.normal(size=d) * 10.0 ** rng.uniform(-3, 3)
        r = r_of(sl, sr, ell=1.0, s_i=1e-12)
        assert r >= 1.0
        assert r_of(sr, sl, ell=1.0, s_i=1e-12) == r          # left and right swap
        c = float(rng.uniform(0.5, 2.0)) * (1 if rng.uniform() < 0.5 else -1)
        r2 = r_of(c * sl, c * sr, ell=1.0, s_i=1e-12)
        assert r2 == r or abs(r2 - r) <= 1e-12 * r


# ---------------------------------------------------------------------------
# the FLAGGED rule through a whole step (1D, one-sided derivatives by hand)
# ---------------------------------------------------------------------------

H = 0.01
N_SIDE = 40          # particles on each side of the centre particle


def _kinked_state():
    """A uniform 1D lattice x_j = j h, j = -40..40, with
      V = 1 + x + 10 x^2    (smooth: one-sided slopes 1 - 10 h and 1 + 10 h at x = 0)
      u = 0                 (at rest: flat)
      P = 1 + 5 |x|         (a kink with a sign change at x = 0)
    The one-sided derivatives of the centre particle (k_side = 1: the nearest
    neighbour on each side) are differences over h:
      V: left (V_0 - V_-1)/h = 1 - 10 h = 0.9, right 1 + 10 h = 1.1
      P: left -5, right +5."""
    j = np.arange(-N_SIDE, N_SIDE + 1)
    x = j * H
    n = x.shape[0]
    V = 1.0 + x + 10.0 * x * x
    P = 1.0 + 5.0 * np.abs(x)
    return {"x": [x], "V": V, "u": [np.zeros(n)], "P": P, "m": H / V,
            "id": np.arange(n, dtype=np.uint32), "n_fluid": n}


def _cfg(limiter):
    return oracle.make_config(1, gamma=1.4, radius_mode=oracle.RADIUS_KSIDE, k_max=8, k_per_side=4, k_side=1,
                              limiter=limiter, s_ref=(0, 0, 0, 0, 0))


def test_flag_from_one_field_gives_every_field_its_phi(oracle_lib):
    st = _kinked_state()
    c = N_SIDE                        # the centre particle, x = 0
    far = 5                           # x = -0.35: every field smooth there
    o = oracle.step(_cfg(oracle.LIM_FLAGGED), st, 1e-4, query=[c, far])
    # centre: r_V = (1.1/0.9 + 0.9/1.1)/2, r_u = 1 (flat), r_P = inf (sign change)
    rV = 0.5 * (1.1 / 0.9 + 0.9 / 1.1)
    assert abs(o["r"][0, 0] - rV) < 1e-12
    assert o["r"][0, 1] == 1.0
    assert np.isinf(o["r"][0, 2])
    assert o["flag"][0] == 1
    # flagged through P alone, yet V and u take phi(r_s), not 1:
    # phi(1) = 1.25, phi(r_V) = 1.25 exp(1 - sqrt(r_V)) (r_V < 3/2), phi(inf) = 0
    assert abs(o["phi"][0, 0] - 1.25 * np.exp(1.0 - np.sqrt(rV))) < 1e-14
    assert abs(o["phi"][0, 1] - 1.25) < 1e-15
    assert o["phi"][0, 2] == 0.0
    # far from the kink: V's slopes differ by 2 h 10 over ~1 - 0.7, r_V < 3/2,
    # P is linear (r = 1), u flat: unflagged, every phi = 1 (pure Lax-Wendroff)
    assert o["flag"][1] == 0
    assert np.all(o["r"][1] <= 1.5)
    assert np.all(o["phi"][1] == 1.0)


def test_paper_mode_applies_phi_everywhere(oracle_lib):
    st = _kinked_state()
    c, far = N_SIDE, 5
    f = oracle.step(_cfg(oracle.LIM_FLAGGED), st, 1e-4, query=[c, far])
    p = oracle.step(_cfg(oracle.LIM_PAPER), st, 1e-4, query=[c, far])
    # the same r; at the flagged particle the same phi
    assert np.array_equal(f["r"], p["r"])
    assert np.array_equal(f["phi"][0], p["phi"][0])
    # away from it PAPER takes phi(r) < 1.25 but != 1 where FLAGGED takes 1
    xV = (-N_SIDE + far) * H
    a, b = 1.0 + 10.0 * (2 * xV - H), 1.0 + 10.0 * (2 * xV + H)   # V's one-sided slopes there
    rV = 0.5 * (b / a + a / b)
    assert abs(p["r"][1, 0] - rV) < 1e-9 * rV
    assert abs(p["phi"][1, 0] - 1.25 * np.exp(1.0 - np.sqrt(rV))) < 1e-9
    assert p["phi"][1, 0] != 1.0


@pytest.mark.parametrize("limiter,expect", [(oracle.LIM_LW, 1.0), (oracle.LIM_UW, 0.0)])
def test_pure_modes_ignore_the_estimator(oracle_lib, limiter, expect):
    o = oracle.step(_cfg(limiter), _kinked_state(), 1e-4, query=[N_SIDE, 5])
    assert np.all(o["phi"] == expect)
    assert o["flag"][0] == 1               # the flag is still reported
