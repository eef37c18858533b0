"""The 2D Yee vortex (Sec. 3: an isentropic vortex convected by a uniform
stream, beta = 5, gamma = 1.4; pressure and velocity errors at t = 8) as a test
of this build's readings of the method in two dimensions.

The vortex starts at (4, 8) in the periodic square [0, 16)^2 on a hexagonal
lattice of spacing dx and is advanced on the GPU (FP32 fits) to t = 8, where
the exact solution is the initial one moved by (8, 0).  Errors are the RMS
(L2) and the maximum (Linf) over the particles of |P - P_exact| and
|u - u_exact|.

Readings this test fixes (the paper does not state them):
  - time step: dt = CFL min_i (m_i V_i)^(1/2) / c_i with CFL 0.4, the local
    spacing from the particle's volume.  The library's own CFL rule takes the
    nearest-neighbour distance, which in a differentially rotating vortex
    collapses as lattice neighbours on nearly equal radii slide past each
    other (at dx = 0.4: from 0.40 to 0.01 by t = 7.5, 381 steps instead of 65);
  - neighbour radius kappa = 2.6 local spacings (18 neighbours on the lattice):
    at kappa = 2.2 the radius lies 3% outside the lattice's third shell, so
    members drift in and out of the stencils as the lattice shears, and the
    errors stop converging.
With these, the Lax-Wendroff scheme (phi = 1) converges at second order from
dx = 0.4 to 0.2 in both norms of both fields, with errors below the paper's.
The full scheme with the state estimator as read (flags where the one-sided
ratio r > 3/2, blend with the axis-sum upwind scheme) does not converge on
this problem: its errors are reported, not bounded.
"""
import os

import numpy as np
import pytest

from paper_2206_11998_gb300 import inputs, lp
from tests.gpu_util import ensure_built

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

L = 16.0
T_END = 8.0
CFL = 0.4


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()


def _paper_table():
    out = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "yee_vortex_errors_paper.txt")):
        if line.strip() and not line.startswith("#"):
            f, dx, l2, li = line.split()
            out[(f, float(dx))] = (float(l2), float(li))
    return out


def run_vortex(dx, limiter, kappa=2.6, k_side=8):
    st = inputs.yee_vortex_2d(dx)
    n = st["V"].shape[0]
    cfg = lp.make_config(2, n, precision=lp.PREC_FP32, kappa=kappa, k_max=40, k_side=k_side, gamma=inputs.YEE_GAMMA,
                         limiter=limiter, periodic=(1, 1, 0), box_lo=(0, 0, 0), box_hi=(L, L, 1),
                         s_ref=inputs.field_scales(st))
    ctx = lp.Context(cfg)
    ps = lp.ParticleSet.from_state(st)
    t, steps = 0.0, 0
    while t < T_END - 1e-12 and steps < 2000:
        c = torch.sqrt(inputs.YEE_GAMMA * ps.P * ps.V)
        dt = CFL * float(torch.min(torch.sqrt(ps.m * ps.V) / c))
        dt = min(dt, T_END - t)
        ctx.step(ps, dt=dt)
        t += dt
        steps += 1
    g = ps.to_state()
    ctx.close()
    rho, u, v, p = inputs.yee_vortex_fields(g["x"][0], g["x"][1], 4.0 + t, 8.0, L)
    eP = g["P"] - p
    eU = np.hypot(g["u"][0] - u, g["u"][1] - v)
    return {"steps": steps, "n": n, "P": (float(np.sqrt(np.mean(eP ** 2))), float(np.abs(eP).max())),
            "u": (float(np.sqrt(np.mean(eU ** 2))), float(eU.max()))}


def test_lax_wendroff_converges_at_second_order_within_the_papers_errors():
    paper = _paper_table()
    res = {dx: run_vortex(dx, lp.LIM_LW) for dx in (0.4, 0.2, 0.1)}
    for dx, r in res.items():
        print("Yee LW dx %.2f: %d particles, %d steps, P L2 %.3g Linf %.3g, u L2 %.3g Linf %.3g"
              % (dx, r["n"], r["steps"], *r["P"], *r["u"]))
    for fld, key in (("P", "pressure"), ("u", "velocity")):
        for dx in (0.4, 0.2):
            l2, li = res[dx][fld]
            pl2, pli = paper[(key, dx)]
            assert l2 < pl2 and li < pli, (fld, dx, (l2, li), (pl2, pli))
        for q in range(2):
            order = np.log2(res[0.4][fld][q] / res[0.2][fld][q])
            assert order > 1.8, (fld, q, order)
    # dx = 0.1: reported (the errors no longer fall at second order there; see DESIGN)
    assert np.isfinite(res[0.1]["P"][0])


def test_full_scheme_errors_are_reported():
    """The estimator and limiter as read, with the upwind one-sided stencils of
    8: the errors at dx = 0.4 and 0.2, and pure upwind for comparison."""
    for lim, name in ((lp.LIM_FLAGGED, "flagged"), (lp.LIM_UW, "upwind")):
        for dx in (0.4, 0.2):
            r = run_vortex(dx, lim)
            print("Yee %s dx %.2f: %d steps, P L2 %.3g Linf %.3g, u L2 %.3g Linf %.3g"
                  % (name, dx, r["steps"], *r["P"], *r["u"]))
