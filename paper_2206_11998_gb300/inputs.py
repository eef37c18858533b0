"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds initial conditions only -- none of the method's arithmetic
(no neighbour radii, fits, rates or updates).  Both the CUDA path and the
oracle read the same float64 arrays produced here.  Random numbers come from
numpy's PCG64 generator with fixed seeds.

A state is a dict::

    x  : list of per-axis float64 arrays (positions)
    V  : float64 specific volume 1/rho
    u  : list of per-axis float64 arrays (velocity)
    P  : float64 pressure
    m  : float64 particle mass
    id : uint32 particle id (0..n-1); ids >= n_fluid are frozen boundary particles
    n_fluid : int
"""
from __future__ import annotations

import numpy as np


def _state(x, V, u, P, m, n_fluid=None):
    n = V.shape[0]
    return {
        "x": [np.ascontiguousarray(a, np.float64) for a in x],
        "V": np.ascontiguousarray(V, np.float64),
        "u": [np.ascontiguousarray(a, np.float64) for a in u],
        "P": np.ascontiguousarray(P, np.float64),
        "m": np.ascontiguousarray(m, np.float64),
        "id": np.arange(n, dtype=np.uint32),
        "n_fluid": int(n if n_fluid is None else n_fluid),
    }


def sod_1d(n_left: int = 889, n_right: int = 111, ghosts: int = 8,
           left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1)):
    """Sod shock tube on [0, 1], discontinuity at 0.5; (rho, u, p) per side.

    Particles sit at cell centres with spacing set by density so that masses are
    (nearly) equal: dx = 0.5 / n_side, m = rho dx (889/111 approximates the 8:1
    density ratio with 1000 particles).  ``ghosts`` frozen particles continue the
    end spacing beyond each end with the end state.
    """
    rl, ul, pl = left
    rr, ur, pr = right
    dxl, dxr = 0.5 / n_left, 0.5 / n_right
    xl = (np.arange(n_left) + 0.5) * dxl
    xr = 0.5 + (np.arange(n_right) + 0.5) * dxr
    gl = -(np.arange(ghosts) + 0.5) * dxl
    gr = 1.0 + (np.arange(ghosts) + 0.5) * dxr
    x = np.concatenate([xl, xr, gl, gr])
    rho = np.concatenate([np.full(n_left, rl), np.full(n_right, rr), np.full(ghosts, rl), np.full(ghosts, rr)])
    u = np.concatenate([np.full(n_left, ul), np.full(n_right, ur), np.full(ghosts, ul), np.full(ghosts, ur)])
    p = np.concatenate([np.full(n_left, pl), np.full(n_right, pr), np.full(ghosts, pl), np.full(ghosts, pr)])
    dx = np.concatenate([np.full(n_left, dxl), np.full(n_right, dxr), np.full(ghosts, dxl), np.full(ghosts, dxr)])
    return _state([x], 1.0 / rho, [u], p, rho * dx, n_fluid=n_left + n_right)


def jittered_lattice_3d(n_side: int = 100, h: float = 0.01, jitter: float = 0.2, seed: int = 1):
    """Cubic lattice of n_side^3 points (cell centres of [0, n_side h)^3) with
    independent uniform jitter in (-jitter h, jitter h) per axis."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = (np.arange(n_side) + 0.5) * h
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()])
    pts = pts + rng.uniform(-jitter * h, jitter * h, size=pts.shape)
    return [np.ascontiguousarray(p) for p in pts]


def random_quadratic_3d(seed: int = 2):
    """Coefficients (c, g, H) of f(x) = c + g.x + x^T H x / 2 with N(0,1) entries
    (H symmetrised)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c = rng.standard_normal()
    g = rng.standard_normal(3)
    A = rng.standard_normal((3, 3))
    H = 0.5 * (A + A.T)
    return float(c), g, H


def quadratic_values(x, c, g, H):
    """Values of the quadratic c + g.x + x^T H x / 2 at positions x (list of 3 arrays)."""
    X = np.stack(x)
    return c + g @ X + 0.5 * np.einsum("in,ij,jn->n", X, H, X)


def gfd_lattice_workload(n_side: int = 100, h: float = 0.01, noise: float = 1e-6,
                         seeds=(1, 2, 3), nfields: int = 1):
    """Jittered lattice plus quadratic fields with additive N(0, noise^2).

    Returns (x, fields, coeffs) where coeffs[f] = (c, g, H) of field f.
    """
    x = jittered_lattice_3d(n_side, h, 0.2, seeds[0])
    fields, coeffs = [], []
    rng = np.random.Generator(np.random.PCG64(seeds[2]))
    for f in range(nfields):
        c, g, H = random_quadratic_3d(seeds[1] + 100 * f)
        v = quadratic_values(x, c, g, H)
        if noise > 0:
            v = v + rng.normal(0.0, noise, size=v.shape)
        fields.append(np.ascontiguousarray(v))
        coeffs.append((c, g, H))
    return x, fields, coeffs


GAS_CLOUD_SIGMA2 = 0.05          # particle positions ~ N(0, 0.05 I)
GAS_CLOUD_GAMMA = 5.0 / 3.0


def gas_cloud_3d(n: int = 2_000_000, seed: int = 4, gamma: float = GAS_CLOUD_GAMMA, r_max_sigma: float = 4.0):
    """Gaussian gas cloud at rest: rho = exp(-r^2/0.1), p = rho^gamma, u = 0.

    Positions are drawn from N(0, 0.05 I) -- the normalised density -- truncated
    to r <= r_max_sigma * sigma (sigma = sqrt(0.05); rejected draws are redrawn
    from the same stream), and every particle carries mass M/n with M the mass of
    the truncated cloud.  The truncation keeps the edge at a density contrast of
    about exp(-r_max_sigma^2 / 2) instead of a handful of far, isolated particles.
    """
    import math
    rng = np.random.Generator(np.random.PCG64(seed))
    sig = np.sqrt(GAS_CLOUD_SIGMA2)
    rmax2 = (r_max_sigma * sig) ** 2 if r_max_sigma else np.inf
    parts, have = [], 0
    while have < n:
        draw = rng.normal(0.0, sig, size=(3, max(1024, int((n - have) * 1.01) + 64)))
        keep = draw[:, (draw * draw).sum(axis=0) <= rmax2]
        parts.append(keep)
        have += keep.shape[1]
    pts = np.concatenate(parts, axis=1)[:, :n]
    r2 = (pts * pts).sum(axis=0)
    rho = np.exp(-r2 / (2.0 * GAS_CLOUD_SIGMA2))
    a = r_max_sigma if r_max_sigma else np.inf
    inside = 1.0 if not np.isfinite(a) else (math.erf(a / math.sqrt(2.0)) -
                                              math.sqrt(2.0 / math.pi) * a * math.exp(-a * a / 2.0))
    M = (2.0 * GAS_CLOUD_SIGMA2 * np.pi) ** 1.5 * inside
    zeros = np.zeros(n)
    return _state([pts[0], pts[1], pts[2]], 1.0 / rho, [zeros, zeros.copy(), zeros.copy()],
                  rho ** gamma, np.full(n, M / n))


def uniform_box_3d(n_side: int = 20, h: float = 0.05, jitter: float = 0.2, seed: int = 7,
                   rho: float = 1.0, p: float = 1.0, vel=(0.0, 0.0, 0.0)):
    """Jittered lattice with a constant state (uniform-flow and Galilean checks)."""
    x = jittered_lattice_3d(n_side, h, jitter, seed)
    n = x[0].shape[0]
    m = np.full(n, rho * h ** 3)
    return _state(x, np.full(n, 1.0 / rho), [np.full(n, float(v)) for v in vel], np.full(n, p), m)


def smooth_wave_3d(n_side: int = 24, h: float = 1.0 / 24, jitter: float = 0.2, seed: int = 9,
                   amp: float = 0.05):
    """Jittered lattice on [0,1)^3 with a smooth, non-trivial state: every field
    varies along every axis (used for step-parity tests)."""
    x = jittered_lattice_3d(n_side, h, jitter, seed)
    X, Y, Z = x
    tp = 2.0 * np.pi
    rho = 1.0 + amp * np.sin(tp * X) * np.cos(tp * Y) + 0.5 * amp * np.sin(tp * Z)
    p = 1.0 + amp * np.cos(tp * X + 0.3) * np.sin(tp * Y + 0.2) * np.cos(tp * Z)
    u = [amp * np.sin(tp * Y + 0.1), amp * np.cos(tp * Z) * np.sin(tp * X), amp * np.sin(tp * (X + Y))]
    m = rho * h ** 3
    return _state(x, 1.0 / rho, u, p, m)


def kh_2d(n: int, amp: float, seed: int, rho_in: float = 2.0, rho_out: float = 1.0,
          vel: float = 0.5, p0: float = 2.5):
    """Doubly periodic Kelvin-Helmholtz shear layer on [0,1)^2.

    rho = 2, u = +0.5 for |y - 0.5| < 0.25; rho = 1, u = -0.5 elsewhere; p = 2.5.
    Particles are placed with number density proportional to rho (equal masses):
    a fraction rho_in * 0.5 / (rho_in * 0.5 + rho_out * 0.5) of them uniformly in
    the strip, the rest uniformly outside it.  v = amp sin(4 pi x) times a
    Gaussian of width 0.05 around each interface.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    f_in = rho_in * 0.5 / (rho_in * 0.5 + rho_out * 0.5)
    n_in = int(round(n * f_in))
    n_out = n - n_in
    xi = rng.uniform(0.0, 1.0, n_in); yi = rng.uniform(0.25, 0.75, n_in)
    xo = rng.uniform(0.0, 1.0, n_out); yo = rng.uniform(0.0, 0.5, n_out)
    yo = np.where(yo < 0.25, yo, yo + 0.5)
    x = np.concatenate([xi, xo]); y = np.concatenate([yi, yo])
    inside = np.abs(y - 0.5) < 0.25
    rho = np.where(inside, rho_in, rho_out)
    u = np.where(inside, vel, -vel)
    s = 0.05
    v = amp * np.sin(4.0 * np.pi * x) * (np.exp(-((y - 0.25) ** 2) / (2 * s * s)) +
                                          np.exp(-((y - 0.75) ** 2) / (2 * s * s)))
    M = rho_in * 0.5 + rho_out * 0.5
    return _state([x, y], 1.0 / rho, [u, v], np.full(n, p0), np.full(n, M / n))


YEE_GAMMA = 1.4
YEE_BETA = 5.0


def yee_vortex_fields(x, y, x0, y0, L, beta=YEE_BETA, gamma=YEE_GAMMA):
    """The isentropic vortex of Sec. 3 (free stream u = 1, v = 0, rho = 1,
    p = 1) centred at (x0, y0), evaluated at (x, y) with the minimum-image
    offsets of a periodic square of edge L:
      T = 1 - (gamma - 1) beta^2 / (8 gamma pi^2) exp(1 - r^2),  rho = T^(1/(gamma-1)),
      u = 1 - beta / (2 pi) exp((1 - r^2)/2) (y - y0),
      v =     beta / (2 pi) exp((1 - r^2)/2) (x - x0),
      p = rho^gamma.
    The printed u line reads e (1 - r^2)/2; it is taken as exp((1 - r^2)/2),
    as in the v line.  Returns (rho, u, v, p)."""
    dx = x - x0
    dy = y - y0
    dx = dx - L * np.round(dx / L)
    dy = dy - L * np.round(dy / L)
    r2 = dx * dx + dy * dy
    T = 1.0 - (gamma - 1.0) * beta ** 2 / (8.0 * gamma * np.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    e = beta / (2.0 * np.pi) * np.exp(0.5 * (1.0 - r2))
    return rho, 1.0 - e * dy, e * dx, rho ** gamma


def yee_vortex_2d(dx: float, L: float = 16.0, x0: float = 4.0, y0: float = 8.0, jitter: float = 0.0, seed: int = 41):
    """Particles of the Yee vortex problem on the periodic square [0, L)^2: a
    hexagonal lattice of spacing dx (rows dx sqrt(3)/2 apart, every other row
    shifted by dx/2), with the row count rounded to an even number so that the
    lattice is periodic in a square (the rows then lie within 1% of the
    hexagonal spacing), optionally jittered by U(-jitter, jitter) dx per axis.
    Each particle carries the mass of its lattice cell at the local density,
    so V = 1/rho holds at t = 0."""
    nx = int(round(L / dx))
    ny = 2 * int(round(L / (dx * np.sqrt(3.0)) ))
    hx, hy = L / nx, L / ny
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    x = ((i + 0.5 + 0.5 * (j % 2)) * hx).ravel()
    y = ((j + 0.5) * hy).ravel()
    if jitter > 0:
        rng = np.random.Generator(np.random.PCG64(seed))
        x = x + jitter * hx * rng.uniform(-1.0, 1.0, x.shape[0])
        y = y + jitter * hy * rng.uniform(-1.0, 1.0, y.shape[0])
    x = np.mod(x, L)
    y = np.mod(y, L)
    rho, u, v, p = yee_vortex_fields(x, y, x0, y0, L)
    return _state([x, y], 1.0 / rho, [u, v], p, rho * hx * hy)


JET_GAMMA = 1.4


def jet_snapshot_3d(n: int = 8_000_000, seed: int = 10, r_jet: float = 1.0, l_jet: float = 12.0,
                    half_width: float = 4.0, length: float = 16.0, density_ratio: float = 1e3,
                    pressure_ratio: float = 100.0, mach: float = 3.0, jitter: float = 0.2):
    """A static snapshot shaped like the supersonic jet: a dense cylinder of gas
    (radius r_jet, along z from 0 to l_jet, rho = 1, p = 1, u_z = mach * c)
    inside an ambient 1/density_ratio as dense at 1/pressure_ratio of the
    pressure, at rest, filling the box [-w, w]^2 x [0, length].

    Equal-mass particles on two jittered cubic lattices: spacing h in the jet
    and h * density_ratio^(1/3) in the ambient (ambient lattice sites closer
    than half their spacing to the cylinder are dropped), with h chosen so that
    about n particles result.  This stands in for the jet's particle state
    until inflow and insertion exist: the same density contrast, so the
    neighbour counts and stencil shapes span the same range.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    v_jet = np.pi * r_jet ** 2 * l_jet
    v_amb = (2.0 * half_width) ** 2 * length - v_jet
    # particles per unit volume: n_jet / v_jet = 1 / h^3, ambient 1 / (h^3 density_ratio)
    h = ((v_jet + v_amb / density_ratio) / n) ** (1.0 / 3.0)
    ha = h * density_ratio ** (1.0 / 3.0)

    def lattice(spacing, lo, hi):
        axes = [np.arange(lo[k] + 0.5 * spacing, hi[k], spacing) for k in range(3)]
        g = np.meshgrid(*axes, indexing="ij")
        return [a.ravel() for a in g]

    jx, jy, jz = lattice(h, (-r_jet, -r_jet, 0.0), (r_jet, r_jet, l_jet))
    keep = jx * jx + jy * jy <= r_jet * r_jet
    jx, jy, jz = jx[keep], jy[keep], jz[keep]
    ax, ay, az = lattice(ha, (-half_width, -half_width, 0.0), (half_width, half_width, length))
    rr = np.sqrt(ax * ax + ay * ay)
    dist = np.where(az <= l_jet, np.maximum(rr - r_jet, 0.0), np.hypot(np.maximum(rr - r_jet, 0.0), az - l_jet))
    keep = dist > 0.5 * ha
    ax, ay, az = ax[keep], ay[keep], az[keep]
    nj, na = jx.shape[0], ax.shape[0]
    x = [np.concatenate([jx, ax]), np.concatenate([jy, ay]), np.concatenate([jz, az])]
    sp = np.concatenate([np.full(nj, h), np.full(na, ha)])
    for k in range(3):
        x[k] = x[k] + sp * rng.uniform(-jitter, jitter, nj + na)
    rho = np.concatenate([np.full(nj, 1.0), np.full(na, 1.0 / density_ratio)])
    p = np.concatenate([np.full(nj, 1.0), np.full(na, 1.0 / pressure_ratio)])
    uz = np.concatenate([np.full(nj, mach * np.sqrt(JET_GAMMA)), np.zeros(na)])
    zero = np.zeros(nj + na)
    return _state(x, 1.0 / rho, [zero, zero.copy(), uz], p, np.full(nj + na, h ** 3))


def jet_inflow_3d(h: float, seed: int = 12, half_width: float = 4.0, length: float = 16.0,
                  density_ratio: float = 1e3, pressure_ratio: float = 100.0, jitter: float = 0.2, fill: float = 1.0):
    """The jet workload with inflow: an ambient gas at rest (rho = 1/density_ratio,
    p = 1/pressure_ratio) filling [-w, w]^2 x [0, length] on a jittered cubic
    lattice of spacing h density_ratio^(1/3), particle mass h^3; a column of
    the jet's gas (rho = 1, p = 1, u_z = 3 c) of radius 1 and height `fill`
    above the inlet on a jittered lattice of spacing h (ambient sites within
    half their spacing of it are dropped); and the parameters of a reservoir
    inlet of radius 1 at the origin, flowing along +z, whose injected particles
    have that same mass on an in-plane lattice of spacing h (a layer of inflow
    at density 1 is then h thick).

    The reservoir (P_res, rho_res) = (2.8^3.5, 2.8^2.5) is the stagnation state
    of a Mach-3 stream at p = 1, rho = 1 (gamma = 1.4: 1 + (gamma - 1) 3^2 / 2 =
    2.8), so an inlet pressure of 1, 100 times the ambient's, draws a Mach-3
    inflow at density 1, 1e3 times the ambient's.  Returns (state, inlet dict)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ha = h * density_ratio ** (1.0 / 3.0)
    axes = [np.arange(-half_width + 0.5 * ha, half_width, ha), np.arange(-half_width + 0.5 * ha, half_width, ha),
            np.arange(0.5 * ha, length, ha)]
    g = np.meshgrid(*axes, indexing="ij")
    xa = [a.ravel() + ha * rng.uniform(-jitter, jitter, a.size) for a in g]
    ra = np.sqrt(xa[0] ** 2 + xa[1] ** 2)
    out = np.maximum(ra - 1.0, 0.0)
    dist = np.where(xa[2] <= fill, out, np.hypot(out, xa[2] - fill))
    keep = dist > 0.5 * ha
    xa = [a[keep] for a in xa]
    axes = [np.arange(-1.0 + 0.5 * h, 1.0, h), np.arange(-1.0 + 0.5 * h, 1.0, h), np.arange(0.5 * h, fill, h)]
    g = np.meshgrid(*axes, indexing="ij")
    xj = [a.ravel() for a in g]
    inside = xj[0] ** 2 + xj[1] ** 2 <= 1.0
    xj = [a[inside] + h * rng.uniform(-jitter, jitter, int(inside.sum())) for a in xj]
    na, nj = xa[0].shape[0], xj[0].shape[0]
    x = [np.concatenate([a, b]) for a, b in zip(xa, xj)]
    n = na + nj
    rho = np.concatenate([np.full(na, 1.0 / density_ratio), np.ones(nj)])
    p = np.concatenate([np.full(na, 1.0 / pressure_ratio), np.ones(nj)])
    uz = np.concatenate([np.zeros(na), np.full(nj, 3.0 * np.sqrt(JET_GAMMA))])
    st = _state(x, 1.0 / rho, [np.zeros(n), np.zeros(n), uz], p, np.full(n, h ** 3))
    inlet = {"center": (0.0, 0.0, 0.0), "axis": 2, "radius": 1.0, "spacing": h, "mass": h ** 3,
             "P_res": 2.8 ** 3.5, "rho_res": 2.8 ** 2.5, "sample_depth": 2.0 * h, "ghost_layers": 3,
             "box": (half_width, 0.5, length)}       # outflow box: |x|, |y| <= w, -0.5 <= z <= length
    return st, inlet


def kh_ensemble_sizes(n_sims: int = 256, lo: int = 10_000, hi: int = 200_000, seed: int = 6):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(lo, hi + 1, size=n_sims)


def kh_ensemble_amplitudes(n_sims: int = 256, base_seed: int = 5):
    return np.array([np.random.Generator(np.random.PCG64(base_seed + k)).uniform(0.01, 0.05)
                     for k in range(n_sims)])


def field_scales(state):
    """Root-mean-square magnitudes used as the estimator's reference scale per
    field (V, u..., P).  Velocity fields that start at rest use the RMS sound
    speed proxy sqrt(P V) as their scale."""
    V, P = state["V"], state["P"]
    cs = float(np.sqrt(np.mean(P * V)))
    out = [float(np.sqrt(np.mean(V * V)))]
    for a in state["u"]:
        r = float(np.sqrt(np.mean(a * a)))
        out.append(r if r > 0 else cs)
    out.append(float(np.sqrt(np.mean(P * P))))
    return out


def take(state, order):
    """State with particles reordered (ids travel with their particles)."""
    out = {k: ([a[order] for a in v] if isinstance(v, list) else
               (v[order] if isinstance(v, np.ndarray) else v)) for k, v in state.items()}
    return out
