"""Write sod_oracle_l1.txt: L1 errors of the oracle's own LP run of the Sod
shock tube (889 + 111 particles, FLAGGED limiter, nearest-neighbour one-sided
stencils, 4 neighbours per side, CFL 0.4) at t = 0.2 against the exact Riemann
solution.  Calls only the oracle."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2206_11998_gb300 import inputs  # noqa: E402


def main():
    st = inputs.sod_1d(889, 111)
    cfg = oracle.make_config(1, gamma=1.4, radius_mode=oracle.RADIUS_KSIDE, k_max=8, k_per_side=4, k_side=1,
                             limiter=oracle.LIM_FLAGGED, s_ref=inputs.field_scales(st), n_fluid=st["n_fluid"])
    t = 0.0
    while t < 0.2 * (1 - 1e-12):
        idx, cnt, tot, d2 = oracle.neighbors(cfg, st["x"], st["V"], st["m"], st["id"])
        dt = min(oracle.cfl_dt(cfg, st["V"], st["P"], st["id"], d2, 0.4), 0.2 - t)
        o = oracle.step(cfg, st, dt)
        st = dict(st, x=o["x"], V=o["V"], u=o["u"], P=o["P"])
        t += dt
    f = st["id"] < st["n_fluid"]
    r, u, p = oracle.riemann_exact(1.4, (1, 0, 1), (0.125, 0, 0.1), 0.5, 0.2, st["x"][0][f])
    e = (np.mean(np.abs(1 / st["V"][f] - r)), np.mean(np.abs(st["u"][0][f] - u)), np.mean(np.abs(st["P"][f] - p)))
    with open(os.path.join(HERE, "sod_oracle_l1.txt"), "w") as fh:
        fh.write("# L1 errors at t = 0.2 of the oracle's Sod run (written by make_sod_golden.py)\n")
        fh.write("rho_l1 %.6e\nu_l1 %.6e\np_l1 %.6e\n" % e)
    print(e)


if __name__ == "__main__":
    main()
