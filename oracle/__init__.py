"""FP64 CPU oracle for the LP hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library in
``paper_2206_11998_gb300``) never imports it and shares no code with it.

Thin ctypes wrapper over ``lp_oracle.c`` (plain FP64 C, no FMA contraction).
Arrays are numpy; positions/fields are lists of per-axis 1-D float64 arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lp_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liblp_oracle.so")
_lock = threading.Lock()
_lib = None

RADIUS_FIXED, RADIUS_VOLUME, RADIUS_KSIDE = 0, 1, 2
LIM_FLAGGED, LIM_PAPER, LIM_LW, LIM_UW = 0, 1, 2, 3
SELECT_NEAREST, SELECT_OCTANT = 0, 1
ST_LINEAR_FALLBACK, ST_NO_FIT, ST_OVERFLOW = 1, 2, 4


def build(force: bool = False) -> str:
    """Compile lp_oracle.c with gcc (FP64, -ffp-contract=off, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class Config(C.Structure):
    """Mirror of ``lpo_config`` in lp_oracle.c."""
    _fields_ = [
        ("dim", C.c_int32), ("radius_mode", C.c_int32),
        ("gamma", C.c_double), ("radius", C.c_double), ("kappa", C.c_double),
        ("k_max", C.c_int32), ("k_side", C.c_int32), ("k_per_side", C.c_int32),
        ("limiter", C.c_int32),
        ("flat_eps", C.c_double), ("active_frac", C.c_double),
        ("s_ref", C.c_double * 5),
        ("periodic", C.c_int32 * 3), ("pad0", C.c_int32),
        ("box_lo", C.c_double * 3), ("box_hi", C.c_double * 3),
        ("rank_tol", C.c_double),
        ("n_fluid", C.c_int64),
        ("select", C.c_int32), ("pad1", C.c_int32),
    ]


def make_config(dim, gamma=1.4, radius_mode=RADIUS_VOLUME, radius=0.0, kappa=2.2, k_max=64,
                k_side=8, k_per_side=4, limiter=LIM_FLAGGED, flat_eps=1e-6, active_frac=0.5,
                s_ref=(0, 0, 0, 0, 0), periodic=(0, 0, 0), box_lo=(0, 0, 0), box_hi=(1, 1, 1),
                rank_tol=1e-12, n_fluid=2**62, select=0) -> Config:
    c = Config()
    c.select = select
    c.dim, c.radius_mode, c.gamma, c.radius, c.kappa = dim, radius_mode, gamma, radius, kappa
    c.k_max, c.k_side, c.k_per_side, c.limiter = k_max, k_side, k_per_side, limiter
    c.flat_eps, c.active_frac, c.rank_tol, c.n_fluid = flat_eps, active_frac, rank_tol, n_fluid
    for k in range(5):
        c.s_ref[k] = float(s_ref[k]) if k < len(s_ref) else 0.0
    for k in range(3):
        c.periodic[k] = int(periodic[k])
        c.box_lo[k] = float(box_lo[k])
        c.box_hi[k] = float(box_hi[k])
    return c


_P = C.c_void_p
_PP = C.POINTER(C.c_void_p)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            L.lpo_morton_keys.argtypes = [C.c_int32, C.c_int64, _PP, _P, C.c_double, C.c_int32, _P]
            L.lpo_neighbors.argtypes = [C.POINTER(Config), C.c_int64, _PP, _P, _P, _P,
                                        C.c_int64, _P, C.c_int32, _P, _P, _P, _P]
            L.lpo_neighbors.restype = C.c_int
            L.lpo_step.argtypes = [C.POINTER(Config), C.c_int64, _PP, _P, _PP, _P, _P, _P,
                                   C.c_double, C.c_int64, _P, _P,
                                   _PP, _P, _PP, _P, _P, _P, _P, _P]
            L.lpo_step.restype = C.c_int
            L.lpo_gfd_central.argtypes = [C.POINTER(Config), _PP, C.c_int32, _PP, C.c_int64, _P,
                                          _P, _P, _P, _P]
            L.lpo_gfd_central.restype = C.c_int
            L.lpo_gfd_onesided.argtypes = [C.POINTER(Config), _PP, C.c_int32, _PP, C.c_int64, _P,
                                           _P, _P, _P]
            L.lpo_gfd_onesided.restype = C.c_int
            L.lpo_cfl_dt.argtypes = [C.POINTER(Config), C.c_int64, _P, _P, _P, _P, C.c_double]
            L.lpo_cfl_dt.restype = C.c_double
            L.lpo_phi.argtypes = [C.c_double]
            L.lpo_phi.restype = C.c_double
            L.lpo_estimator_r.argtypes = [C.c_int32, _P, _P] + [C.c_double] * 5
            L.lpo_inflow_state.argtypes = [C.c_double] * 4 + [_P, _P]
            L.lpo_free_surface_ghosts.argtypes = [C.POINTER(Config), C.c_int64, _PP, _P, _PP, _P, _P, C.c_int32,
                                                  C.c_double, C.c_uint32, C.c_int64, _PP, _P, _PP, _P, _P, _P]
            L.lpo_free_surface_ghosts.restype = C.c_int64
            L.lpo_estimator_r.restype = C.c_double
            L.lpo_riemann_star.argtypes = [C.c_double] * 7 + [_P, _P]
            L.lpo_riemann_star.restype = C.c_int
            L.lpo_riemann_exact.argtypes = [C.c_double] * 9 + [C.c_int64, _P, _P, _P, _P]
            L.lpo_features.argtypes = [C.POINTER(Config), C.c_int64, _PP, _P, _PP, _P, _P, _P, C.c_int64, _P, _P]
            L.lpo_features.restype = C.c_int
            L.lpo_mlp_forward.argtypes = [C.c_int64, _P, _P, _P, _P, C.c_double, _P, _P]
            L.lpo_mlp_loss_grad.argtypes = [C.c_int64, _P, _P, C.c_double, _P, _P, _P, C.c_double,
                                            _P, _P, _P, _P]
            L.lpo_mlp_loss_grad.restype = C.c_double
            L.lpo_adam.argtypes = [C.c_int64, _P, _P, _P, _P, C.c_int64, C.c_double, C.c_double,
                                   C.c_double, C.c_double]
            L.lpo_num_threads.restype = C.c_int
            L.lpo_set_num_threads.argtypes = [C.c_int]
            _lib = L
    return _lib


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _ptrs(arrs):
    arr = (C.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
    return C.cast(arr, _PP), arr


def num_threads() -> int:
    return int(lib().lpo_num_threads())


def set_num_threads(t: int) -> None:
    lib().lpo_set_num_threads(int(t))


# ---------------------------------------------------------------------------
# public oracle functions
# ---------------------------------------------------------------------------

def morton_keys(x, lo, L, bits):
    """Morton keys (uint64) of positions x (list of per-axis arrays)."""
    dim = len(x)
    xs = [_c(a, np.float64) for a in x]
    n = xs[0].shape[0]
    lo_a = _c(list(lo) + [0.0] * (3 - len(lo)), np.float64)
    out = np.zeros(n, np.uint64)
    px, keep = _ptrs(xs)
    lib().lpo_morton_keys(dim, n, px, _ptr(lo_a), float(L), int(bits), _ptr(out))
    return out


def neighbors(cfg: Config, x, V, m, ids, query=None, window=True):
    """Neighbour lists (input indices), counts, totals and d2 of the nearest."""
    xs = [_c(a, np.float64) for a in x]
    V = _c(V, np.float64); m = _c(m, np.float64); ids = _c(ids, np.uint32)
    n = V.shape[0]
    q = np.arange(n, dtype=np.int64) if query is None else _c(query, np.int64)
    nq = q.shape[0]
    cnt = np.zeros(nq, np.uint32); tot = np.zeros(nq, np.uint32)
    idx = np.zeros((nq, cfg.k_max), np.int64); d2 = np.zeros(nq, np.float64)
    px, keep = _ptrs(xs)
    rc = lib().lpo_neighbors(C.byref(cfg), n, px, _ptr(V), _ptr(m), _ptr(ids), nq, _ptr(q),
                             1 if window else 0, _ptr(cnt), _ptr(tot), _ptr(idx), _ptr(d2))
    if rc != 0:
        raise MemoryError("lpo_neighbors failed")
    return idx, cnt, tot, d2


def gfd_central(cfg: Config, x, fields, cnt, idx, query=None):
    """Central second-order GFD derivatives: array [nf, nq, n_u] and status."""
    xs = [_c(a, np.float64) for a in x]
    Fs = [_c(a, np.float64) for a in fields]
    n = xs[0].shape[0]
    q = np.arange(n, dtype=np.int64) if query is None else _c(query, np.int64)
    nq = q.shape[0]
    nu = {1: 2, 2: 5, 3: 9}[cfg.dim]
    out = np.zeros((len(Fs), nq, nu), np.float64)
    st = np.zeros(nq, np.uint32)
    px, k1 = _ptrs(xs); pf, k2 = _ptrs(Fs)
    cnt = _c(cnt, np.uint32); idx = _c(idx, np.int64)
    rc = lib().lpo_gfd_central(C.byref(cfg), px, len(Fs), pf, nq, _ptr(q), _ptr(cnt), _ptr(idx),
                               _ptr(out), _ptr(st))
    if rc != 0:
        raise ValueError("lpo_gfd_central failed")
    return out, st


def gfd_onesided(cfg: Config, x, fields, cnt, idx, query=None):
    """One-sided first derivatives: array [nq, dim, 2 (left, right), nf]."""
    xs = [_c(a, np.float64) for a in x]
    Fs = [_c(a, np.float64) for a in fields]
    n = xs[0].shape[0]
    q = np.arange(n, dtype=np.int64) if query is None else _c(query, np.int64)
    nq = q.shape[0]
    out = np.zeros((nq, cfg.dim, 2, len(Fs)), np.float64)
    px, k1 = _ptrs(xs); pf, k2 = _ptrs(Fs)
    cnt = _c(cnt, np.uint32); idx = _c(idx, np.int64)
    rc = lib().lpo_gfd_onesided(C.byref(cfg), px, len(Fs), pf, nq, _ptr(q), _ptr(cnt), _ptr(idx),
                                _ptr(out))
    if rc != 0:
        raise ValueError("lpo_gfd_onesided failed")
    return out


def cfl_dt(cfg: Config, V, P, ids, d2min, cfl):
    V = _c(V, np.float64); P = _c(P, np.float64); ids = _c(ids, np.uint32)
    d2min = _c(d2min, np.float64)
    return float(lib().lpo_cfl_dt(C.byref(cfg), V.shape[0], _ptr(V), _ptr(P), _ptr(ids),
                                  _ptr(d2min), float(cfl)))


def free_surface_ghosts(cfg: Config, state: dict, min_per_side=1, p_ghost=0.0, ghost_base=2**31):
    """Ghost particles completing the free-surface neighbourhoods of the fluid
    particles of ``state`` (Sec. 2.2 step 3; lpo_free_surface_ghosts): a state
    dict (x, V, u, P, m, id) of the ghosts, in (particle, axis, side) order."""
    dim = cfg.dim
    xs = [_c(a, np.float64) for a in state["x"]]
    us = [_c(a, np.float64) for a in state["u"]]
    V = _c(state["V"], np.float64); m = _c(state["m"], np.float64); ids = _c(state["id"], np.uint32)
    n = V.shape[0]
    cap = 2 * dim * n
    ox = [np.zeros(cap) for _ in range(dim)]
    ou = [np.zeros(cap) for _ in range(dim)]
    oV = np.zeros(cap); oP = np.zeros(cap); om = np.zeros(cap); oid = np.zeros(cap, np.uint32)
    px, k1 = _ptrs(xs); pu, k2 = _ptrs(us); pox, k3 = _ptrs(ox); pou, k4 = _ptrs(ou)
    ng = lib().lpo_free_surface_ghosts(C.byref(cfg), n, px, _ptr(V), pu, _ptr(m), _ptr(ids), int(min_per_side),
                                       float(p_ghost), int(ghost_base), cap, pox, _ptr(oV), pou, _ptr(oP),
                                       _ptr(om), _ptr(oid))
    if ng < 0:
        raise MemoryError("lpo_free_surface_ghosts failed")
    return {"x": [a[:ng] for a in ox], "V": oV[:ng], "u": [a[:ng] for a in ou], "P": oP[:ng], "m": om[:ng],
            "id": oid[:ng]}


def step(cfg: Config, state: dict, dt: float, query=None, forced_phi=None):
    """One LP step for the query particles (all by default).

    ``state``: dict with x (list of arrays), V, u (list), P, m, id.
    Returns dict with x, V, u, P (new values of the queries), flag, phi, r, status.
    """
    dim = cfg.dim
    xs = [_c(a, np.float64) for a in state["x"]]
    us = [_c(a, np.float64) for a in state["u"]]
    V = _c(state["V"], np.float64); P = _c(state["P"], np.float64)
    m = _c(state["m"], np.float64); ids = _c(state["id"], np.uint32)
    n = V.shape[0]
    q = np.arange(n, dtype=np.int64) if query is None else _c(query, np.int64)
    nq = q.shape[0]
    nf = dim + 2
    xn = [np.zeros(nq) for _ in range(dim)]
    un = [np.zeros(nq) for _ in range(dim)]
    Vn = np.zeros(nq); Pn = np.zeros(nq)
    flag = np.zeros(nq, np.uint8)
    phi = np.zeros((nq, nf)); rr = np.zeros((nq, nf)); st = np.zeros(nq, np.uint32)
    fp = None
    if forced_phi is not None:
        fp = _c(forced_phi, np.float64)
        assert fp.shape == (nq, nf)
    px, k1 = _ptrs(xs); pu, k2 = _ptrs(us); pxn, k3 = _ptrs(xn); pun, k4 = _ptrs(un)
    rc = lib().lpo_step(C.byref(cfg), n, px, _ptr(V), pu, _ptr(P), _ptr(m), _ptr(ids), float(dt),
                        nq, _ptr(q), _ptr(fp) if fp is not None else None,
                        pxn, _ptr(Vn), pun, _ptr(Pn), _ptr(flag), _ptr(phi), _ptr(rr), _ptr(st))
    if rc != 0:
        raise MemoryError("lpo_step failed")
    return {"x": xn, "V": Vn, "u": un, "P": Pn, "flag": flag, "phi": phi, "r": rr, "status": st}


def features(cfg: Config, state: dict, query=None):
    """The learned estimator's eight inputs for the query particles: [nq, 8]."""
    xs = [_c(a, np.float64) for a in state["x"]]
    us = [_c(a, np.float64) for a in state["u"]]
    V = _c(state["V"], np.float64); P = _c(state["P"], np.float64)
    m = _c(state["m"], np.float64); ids = _c(state["id"], np.uint32)
    n = V.shape[0]
    q = np.arange(n, dtype=np.int64) if query is None else _c(query, np.int64)
    out = np.zeros((q.shape[0], 8))
    px, k1 = _ptrs(xs); pu, k2 = _ptrs(us)
    rc = lib().lpo_features(C.byref(cfg), n, px, _ptr(V), pu, _ptr(P), _ptr(m), _ptr(ids), q.shape[0], _ptr(q),
                            _ptr(out))
    if rc != 0:
        raise MemoryError("lpo_features failed")
    return out


def phi(r: float) -> float:
    return float(lib().lpo_phi(float(r)))


def estimator_r(sl, sr, ell, s_i, s_ref=0.0, flat_eps=1e-6, active_frac=0.5) -> float:
    """State estimator r of one field from its left/right one-sided derivatives
    along each axis (sl[k], sr[k]), the nearest-neighbour distance ell and the
    particle's value s_i."""
    sl = _c(sl, np.float64); sr = _c(sr, np.float64)
    assert sl.shape == sr.shape and 1 <= sl.shape[0] <= 3
    return float(lib().lpo_estimator_r(sl.shape[0], _ptr(sl), _ptr(sr), float(ell), float(s_i), float(s_ref),
                                       float(flat_eps), float(active_frac)))


def inflow_state(gamma, P_res, rho_res, P_inf):
    """(rho_inf, u_inf) of particles entering from a reservoir at rest."""
    r = np.zeros(1); u = np.zeros(1)
    lib().lpo_inflow_state(float(gamma), float(P_res), float(rho_res), float(P_inf), _ptr(r), _ptr(u))
    return float(r[0]), float(u[0])


def riemann_star(gamma, left, right):
    """(p*, u*) of the Riemann problem with left/right = (rho, u, p)."""
    ps = np.zeros(1); us = np.zeros(1)
    lib().lpo_riemann_star(float(gamma), *map(float, left), *map(float, right), _ptr(ps), _ptr(us))
    return float(ps[0]), float(us[0])


def riemann_exact(gamma, left, right, x0, t, xs):
    xs = _c(xs, np.float64)
    n = xs.shape[0]
    r = np.zeros(n); u = np.zeros(n); p = np.zeros(n)
    lib().lpo_riemann_exact(float(gamma), *map(float, left), *map(float, right), float(x0),
                            float(t), n, _ptr(xs), _ptr(r), _ptr(u), _ptr(p))
    return r, u, p


MLP_IN, MLP_H = 8, 32


def mlp_forward(X, W1, b1, w2, b2):
    X = _c(X, np.float64); W1 = _c(W1, np.float64); b1 = _c(b1, np.float64)
    w2 = _c(w2, np.float64)
    n = X.shape[0]
    z = np.zeros(n); p = np.zeros(n)
    lib().lpo_mlp_forward(n, _ptr(X), _ptr(W1), _ptr(b1), _ptr(w2), float(b2), _ptr(z), _ptr(p))
    return z, p


def mlp_loss_grad(X, y, pos_weight, W1, b1, w2, b2):
    X = _c(X, np.float64); y = _c(y, np.float64); W1 = _c(W1, np.float64)
    b1 = _c(b1, np.float64); w2 = _c(w2, np.float64)
    n = X.shape[0]
    gW1 = np.zeros((MLP_H, MLP_IN)); gb1 = np.zeros(MLP_H); gw2 = np.zeros(MLP_H); gb2 = np.zeros(1)
    L = lib().lpo_mlp_loss_grad(n, _ptr(X), _ptr(y), float(pos_weight), _ptr(W1), _ptr(b1),
                                _ptr(w2), float(b2), _ptr(gW1), _ptr(gb1), _ptr(gw2), _ptr(gb2))
    return float(L), gW1, gb1, gw2, float(gb2[0])


def adam(w, g, mo, ve, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam update of float64 arrays w, mo, ve."""
    for a in (w, mo, ve):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _c(g, np.float64)
    lib().lpo_adam(w.size, _ptr(w), _ptr(g), _ptr(mo), _ptr(ve), int(t), float(lr), float(beta1),
                   float(beta2), float(eps))
