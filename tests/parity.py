"""Parity harness of the GPU step tests: the ambiguity band of the estimator's
discontinuous decisions, and the field and rate comparisons.

The state estimator (Sec. 2.1) takes discrete decisions from continuous
values: the sign of s_l s_r (r = inf on a sign change), which axes are active
(max(|s_l|, |s_r|) against active_frac of the largest), whether a field is
flat (max|d| ell against flat_eps max(|s|, s_ref)), and the flag (some r_s >
3/2).  Where the GPU's and the oracle's arithmetic straddle a threshold they
may decide differently.  Such a particle is accepted only when the oracle's
own FP64 values put one of its decisions inside the band:

  |r_s - 3/2| < band_r            for some field s, or
  margin < band_rel               for a sign (min(|s_l|, |s_r|) / G_s), an
                                  activity test (|g_k - active_frac G_s| / G_s)
                                  or a flatness test (|G_s ell - flat_eps S_s| /
                                  (flat_eps S_s)) of some field,

with G_s the largest one-sided magnitude of field s over the axes.  The bands:
  FP64 path: band_r = 1e-6, band_rel = 1e-10.  The GPU's FP64 one-sided
      derivatives agree with the oracle's to ~cond u ~ 1e-14 relative to G.
  FP32 path: band_r = band_rel = 1e-3.  FP32 one-sided derivatives carry a
      relative error of ~cond u with u = 6e-8 and cond <= 1 / tau32 = 1e3 (a
      stencil worse than that is redone in FP64): <= 6e-5 relative to G; r =
      (a/b + b/a)/2 near 3/2 moves by about 4 times that, 2.4e-4.  The bands
      are 4x and 16x those worst cases.
For the particles accepted, the oracle is run again with the GPU's phi forced.
"""
import numpy as np

import oracle
from paper_2206_11998_gb300 import lp

BANDS = {lp.PREC_FP64: (1e-6, 1e-10), lp.PREC_FP32: (1e-3, 1e-3)}


def decision_margins(ocfg, st, q, r_oracle):
    """Smallest margin of the estimator decisions of the query particles q
    (indices into st), from the oracle's FP64 one-sided derivatives.  Returns
    (r margin, relative margin) arrays of length len(q)."""
    q = np.asarray(q, np.int64)
    dim = ocfg.dim
    oidx, ocnt, _, od2 = oracle.neighbors(ocfg, st["x"], st["V"], st["m"], st["id"], query=q)
    fields = [st["V"]] + list(st["u"][:dim]) + [st["P"]]
    os_ = oracle.gfd_onesided(ocfg, st["x"], fields, ocnt, oidx, query=q)      # [nq, dim, 2, nf]
    ell = np.sqrt(od2)
    nq, nf = len(q), dim + 2
    m_rel = np.full(nq, np.inf)
    for f in range(nf):
        sl, sr = os_[:, :, 0, f], os_[:, :, 1, f]
        g = np.maximum(np.abs(sl), np.abs(sr))                  # [nq, dim]
        G = g.max(axis=1)
        S = np.maximum(np.abs(fields[f][q]), ocfg.s_ref[f])
        floor = ocfg.flat_eps * S
        with np.errstate(divide="ignore", invalid="ignore"):
            flat = np.where(floor > 0, np.abs(G * ell - floor) / floor, np.where(G * ell > 0, np.inf, 0.0))
            m_rel = np.minimum(m_rel, flat)
            Gs = np.where(G > 0, G, np.inf)
            act = np.abs(g - ocfg.active_frac * G[:, None]) / Gs[:, None]
            sgn = np.minimum(np.abs(sl), np.abs(sr)) / Gs[:, None]
        live = G * ell > floor                                  # decisions below the floor do not count
        act = np.where(live[:, None], act, np.inf)
        # a sign decision counts on an axis that is active or at the activity threshold
        near_active = g >= ocfg.active_frac * G[:, None] * (1.0 - 1e-3)
        sgn = np.where(live[:, None] & near_active, sgn, np.inf)
        m_rel = np.minimum(m_rel, np.minimum(act.min(axis=1), sgn.min(axis=1)))
    r = np.asarray(r_oracle, np.float64)
    with np.errstate(invalid="ignore"):
        m_r = np.where(np.isfinite(r), np.abs(r - 1.5), np.inf).min(axis=1)
    return m_r, m_rel


def resolve(ocfg, st, q, prec, g_flag, g_phi, o, dt, max_diff, forced=None):
    """Compare the GPU's discrete decisions (flag and phi of the query particles
    q, in the order of q) with the oracle's step output o for q; particles that
    differ must lie in the band, and there may be at most max_diff of them.
    forced (optional, [len(q), nf], NaN = free): phi the oracle run o was given
    already (the learned gate's decisions); those particles are not compared.
    Returns (oracle output with the GPU's phi forced where needed, number of
    ambiguous particles)."""
    q = np.asarray(q, np.int64)
    free = np.ones(len(q), bool) if forced is None else ~np.isfinite(forced).any(axis=1)
    diff = np.nonzero(free & ((g_flag != o["flag"]) | (np.abs(g_phi - o["phi"]).max(axis=1) > 1e-3)))[0]
    if len(diff) == 0:
        return o, 0
    assert len(diff) <= max_diff, "%d decisions differ" % len(diff)
    band_r, band_rel = BANDS[prec]
    qq = q[diff]
    m_r, m_rel = decision_margins(ocfg, st, qq, o["r"][diff])
    inside = (m_r < band_r) | (m_rel < band_rel)
    assert inside.all(), ("decisions differ outside the band", list(zip(qq[~inside], m_r[~inside],
                                                                        m_rel[~inside])))
    forced = np.full(o["phi"].shape, np.nan) if forced is None else forced.copy()
    forced[diff] = g_phi[diff]
    return oracle.step(ocfg, st, dt, query=q, forced_phi=forced), len(diff)


def normwise(g, o):
    """max |g - o| / max |o| (per-field normwise relative error)."""
    den = np.abs(o).max()
    num = np.abs(g - o).max()
    return num / den if den > 0 else num


def field_and_rate_errors(dim, s0, g, o, dt):
    """Normwise errors of the new state and of the rates (s^{n+1} - s^n) / dt
    per field: s0, g, o are dicts with V, u (list), P, x (list) of one particle
    set in the same order."""
    errs, rates = {}, {}
    names = ["V"] + ["u%d" % k for k in range(dim)] + ["P"]
    get = lambda d, nm: d[nm] if nm in ("V", "P") else d["u"][int(nm[1])]
    for nm in names:
        a0, ga, oa = get(s0, nm), get(g, nm), get(o, nm)
        errs[nm] = normwise(ga, oa)
        rates[nm] = normwise((ga - a0) / dt, (oa - a0) / dt)
    for k in range(dim):
        errs["x%d" % k] = normwise(g["x"][k], o["x"][k])
    return errs, rates
