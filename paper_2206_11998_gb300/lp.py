"""ctypes binding of liblp.so (declared in include/lp.h).

Argument marshalling only: every step of the LP hot path runs in the CUDA
library.  PyTorch provides device memory (torch.cuda tensors) and streams.
There is no CPU fallback: if liblp.so is missing or cannot be loaded, every
call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblp.so")

OK, ERR_ARG, ERR_CUDA, ERR_CAPACITY, ERR_ILLCOND, ERR_NONFINITE, ERR_TIMEOUT, ERR_STATE = range(8)
PREC_FP32, PREC_FP64 = 0, 1
RADIUS_FIXED, RADIUS_VOLUME, RADIUS_KSIDE = 0, 1, 2
LIM_FLAGGED, LIM_PAPER, LIM_LW, LIM_UW = 0, 1, 2, 3
EST_PLAIN, EST_MLP = 0, 1
OUT_F32, OUT_F64 = 0, 1
REFINE_AUTO, REFINE_ALWAYS, REFINE_NEVER = 0, 1, 2
SELECT_NEAREST, SELECT_OCTANT = 0, 1
SCHED_FUSED, SCHED_SPLIT, SCHED_QUERY_WARP, SCHED_QUEUE_QUERY, SCHED_QUEUE_FIT = 0, 1, 2, 4, 8
AUTOTUNE_TIMES = 6

EXPORTED = [
    "lp_create", "lp_destroy", "lp_build_neighbors", "lp_gfd_derivs", "lp_onesided_derivs", "lp_step",
    "lp_export_neighbors", "lp_grid_info", "lp_dt_device", "lp_get_stats", "lp_reset_stats",
    "lp_status_string", "lp_version", "lp_set_profiling", "lp_phase_times", "lp_phase_name",
    "lp_sort_keys_noalloc", "lp_mlp_set_params", "lp_mlp_get_params", "lp_mlp_grad", "lp_mlp_adam_step",
    "lp_mlp_train", "lp_mlp_infer", "lp_step_batched", "lp_graph_capture", "lp_graph_launch",
    "lp_set_schedule", "lp_get_schedule", "lp_autotune", "lp_step_host", "lp_inflow", "lp_reserve",
    "lp_remove_outside", "lp_free_surface_ghosts", "lp_remove_ghosts", "lp_octant_coverage",
]
MLP_IN, MLP_H = 8, 32
MLP_NPARAM = MLP_H * MLP_IN + MLP_H + MLP_H + 1
NOALLOC_MAX_N = 262144
NPHASES = 10


class LPError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = "%s: %s (%d)" % (where, _lib_or_none_status(code), code)
        super().__init__(msg)


class Config(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("precision", C.c_int32), ("radius_mode", C.c_int32), ("k_max", C.c_int32),
        ("k_side", C.c_int32), ("k_per_side", C.c_int32), ("limiter", C.c_int32), ("estimator", C.c_int32),
        ("gamma", C.c_double), ("radius", C.c_double), ("kappa", C.c_double), ("flat_eps", C.c_double),
        ("active_frac", C.c_double), ("s_ref", C.c_double * 5), ("tau32", C.c_double), ("tau64", C.c_double),
        ("periodic", C.c_int32 * 3), ("max_level", C.c_int32),
        ("box_lo", C.c_double * 3), ("box_hi", C.c_double * 3),
        ("n_fluid", C.c_int64), ("capacity", C.c_int64),
        ("mlp_tau_lo", C.c_double), ("mlp_audit", C.c_int32), ("max_sims", C.c_int32),
        ("refine", C.c_int32), ("refine_ratio", C.c_double),
        ("select", C.c_int32), ("reserved", C.c_int32), ("t_end", C.c_double),
    ]


class Particles(C.Structure):
    _fields_ = [("n", C.c_int64), ("x", C.c_void_p * 3), ("V", C.c_void_p), ("u", C.c_void_p * 3),
                ("P", C.c_void_p), ("m", C.c_void_p), ("id", C.c_void_p)]


class Neighbors(C.Structure):
    _fields_ = [("n", C.c_int64), ("k_max", C.c_int32), ("pad", C.c_int32), ("count", C.c_void_p),
                ("total", C.c_void_p), ("idx", C.c_void_p), ("d2min", C.c_void_p), ("keys", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("dt", C.c_double), ("steps", C.c_int64), ("n_flagged", C.c_int64),
                ("n_fp64_redo", C.c_int64), ("n_linear", C.c_int64), ("n_nofit", C.c_int64),
                ("n_overflow", C.c_int64), ("n_nonfinite", C.c_int64), ("n_mlp_uncertain", C.c_int64),
                ("max_count", C.c_uint32), ("status", C.c_uint32), ("kernel_launches", C.c_int64),
                ("n_mlp_skip", C.c_int64), ("n_mlp_miss", C.c_int64), ("n_query_fallback", C.c_int64),
                ("n_refined", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class StepDiag(C.Structure):
    _fields_ = [("flag", C.c_void_p), ("phi", C.c_void_p), ("r", C.c_void_p), ("features", C.c_void_p),
                ("gate_p", C.c_void_p)]


class Inlet(C.Structure):
    _fields_ = [("center", C.c_double * 3), ("axis", C.c_int32), ("ghost_layers", C.c_int32),
                ("radius", C.c_double), ("spacing", C.c_double), ("mass", C.c_double),
                ("P_res", C.c_double), ("rho_res", C.c_double), ("sample_depth", C.c_double),
                ("first_id", C.c_uint32), ("ghost_id", C.c_uint32)]


class InflowInfo(C.Structure):
    _fields_ = [("P_inf", C.c_double), ("rho_inf", C.c_double), ("u_inf", C.c_double), ("c_inf", C.c_double),
                ("h_z", C.c_double), ("travel", C.c_double), ("layers", C.c_int64), ("layers_total", C.c_int64),
                ("npat", C.c_int64), ("sampled", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def make_inlet(center, axis, radius, spacing, mass, P_res, rho_res, sample_depth, ghost_layers=2, first_id=0,
               ghost_id=2**31) -> Inlet:
    """A reservoir inlet for Context.inflow (see lp_inflow in lp.h)."""
    q = Inlet()
    for k in range(3):
        q.center[k] = float(center[k])
    q.axis, q.ghost_layers = int(axis), int(ghost_layers)
    q.radius, q.spacing, q.mass = float(radius), float(spacing), float(mass)
    q.P_res, q.rho_res, q.sample_depth = float(P_res), float(rho_res), float(sample_depth)
    q.first_id, q.ghost_id = int(first_id), int(ghost_id)
    return q


def _diag(flag, phi, r, features, gate_p):
    d = StepDiag()
    d.flag, d.phi, d.r, d.features, d.gate_p = _ptr(flag), _ptr(phi), _ptr(r), _ptr(features), _ptr(gate_p)
    return d


_lib = None


def _lib_or_none_status(code):
    try:
        return lib().lp_status_string(code).decode()
    except Exception:
        return "status"


def lib():
    """Load liblp.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("liblp.so not found at %s; build it with paper_2206_11998_gb300.build.build()"
                               % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        L.lp_create.argtypes = [C.POINTER(Config), C.POINTER(C.c_void_p)]
        L.lp_destroy.argtypes = [P]
        L.lp_build_neighbors.argtypes = [P, C.POINTER(Particles), C.POINTER(Neighbors), P]
        L.lp_gfd_derivs.argtypes = [P, C.POINTER(Particles), C.POINTER(C.c_void_p), C.c_int32, C.c_int32, P, P, P]
        L.lp_onesided_derivs.argtypes = [P, C.POINTER(Particles), C.POINTER(C.c_void_p), C.c_int32, P, P]
        L.lp_step.argtypes = [P, C.POINTER(Particles), C.c_double, C.c_double, P, C.POINTER(StepDiag), P]
        L.lp_step_host.argtypes = [P, C.POINTER(Particles), C.c_double, C.c_double, P, C.POINTER(StepDiag), P]
        L.lp_step_host.restype = C.c_int
        L.lp_step_batched.argtypes = [P, C.POINTER(Particles), P, C.c_int32, C.c_double, C.c_double, P,
                                      C.POINTER(StepDiag), P]
        L.lp_step_batched.restype = C.c_int
        L.lp_graph_capture.argtypes = [P, C.POINTER(Particles), P, C.c_int32, C.c_double, C.c_double, P, P]
        L.lp_graph_capture.restype = C.c_int
        L.lp_graph_launch.argtypes = [P, P]
        L.lp_set_schedule.argtypes = [P, C.c_int32]
        L.lp_get_schedule.argtypes = [P, P]
        L.lp_autotune.argtypes = [P, C.POINTER(Particles), P, C.c_int32, C.c_double, C.c_double, C.c_int32, P, P]
        L.lp_graph_launch.restype = C.c_int
        L.lp_export_neighbors.argtypes = [P, P, P, P, P, P, P]
        L.lp_grid_info.argtypes = [P, P, P]
        L.lp_dt_device.argtypes = [P]
        L.lp_dt_device.restype = C.c_void_p
        L.lp_get_stats.argtypes = [P, C.POINTER(Stats), P]
        L.lp_reset_stats.argtypes = [P, P]
        L.lp_status_string.argtypes = [C.c_int]
        L.lp_status_string.restype = C.c_char_p
        L.lp_version.restype = C.c_char_p
        L.lp_set_profiling.argtypes = [P, C.c_int32]
        L.lp_phase_times.argtypes = [P, P, P, P]
        L.lp_phase_name.argtypes = [C.c_int32]
        L.lp_phase_name.restype = C.c_char_p
        L.lp_sort_keys_noalloc.argtypes = [C.c_int32, C.c_int64, P, P, P, P, P, P]
        L.lp_sort_keys_noalloc.restype = C.c_int
        L.lp_mlp_set_params.argtypes = [P, P]
        L.lp_mlp_get_params.argtypes = [P, P, P]
        L.lp_mlp_grad.argtypes = [P, P, P, C.c_int64, C.c_double, P, P, P]
        L.lp_mlp_adam_step.argtypes = [P, P, C.c_double, P]
        L.lp_mlp_train.argtypes = [P, P, P, C.c_int64, C.c_int32, C.c_int32, C.c_double, C.c_double, P, P]
        L.lp_mlp_infer.argtypes = [P, P, C.c_int64, P, P]
        L.lp_inflow.argtypes = [P, C.POINTER(Particles), C.c_int64, C.POINTER(Inlet), C.POINTER(C.c_int64),
                                C.POINTER(InflowInfo), P]
        L.lp_inflow.restype = C.c_int
        L.lp_reserve.argtypes = [P, C.c_int64]
        L.lp_remove_outside.argtypes = [P, C.POINTER(Particles), P, P, C.POINTER(C.c_int64), P]
        L.lp_remove_outside.restype = C.c_int
        L.lp_reserve.restype = C.c_int
        L.lp_free_surface_ghosts.argtypes = [P, C.POINTER(Particles), C.c_int64, C.c_int32, C.c_double, C.c_uint32,
                                             C.POINTER(C.c_int64), P]
        L.lp_free_surface_ghosts.restype = C.c_int
        L.lp_remove_ghosts.argtypes = [P, C.POINTER(Particles), C.c_uint32, C.POINTER(C.c_int64), P]
        L.lp_remove_ghosts.restype = C.c_int
        L.lp_octant_coverage.argtypes = [P, P, C.POINTER(C.c_int64), P]
        L.lp_octant_coverage.restype = C.c_int
        for name in ("lp_mlp_set_params", "lp_mlp_get_params", "lp_mlp_grad", "lp_mlp_adam_step", "lp_mlp_train",
                     "lp_mlp_infer"):
            getattr(L, name).restype = C.c_int
        for name in ("lp_create", "lp_destroy", "lp_build_neighbors", "lp_gfd_derivs", "lp_onesided_derivs",
                     "lp_step", "lp_export_neighbors", "lp_grid_info", "lp_get_stats", "lp_reset_stats",
                     "lp_set_profiling", "lp_phase_times"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(rc, where):
    if rc != OK:
        raise LPError(rc, where)


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def make_config(dim, capacity, precision=PREC_FP32, radius_mode=RADIUS_VOLUME, radius=0.0, kappa=2.2,
                k_max=64, k_side=8, k_per_side=4, gamma=1.4, limiter=LIM_FLAGGED, estimator=EST_PLAIN,
                flat_eps=1e-6, active_frac=0.5, s_ref=(0, 0, 0, 0, 0), tau32=1e-3, tau64=1e-12,
                periodic=(0, 0, 0), box_lo=(0, 0, 0), box_hi=(1, 1, 1), n_fluid=2**62, max_level=0,
                mlp_tau_lo=0.05, mlp_audit=0, max_sims=1, refine=0, refine_ratio=0.1, select=0,
                t_end=0.0) -> Config:
    c = Config()
    c.select = select
    c.t_end = t_end
    c.dim, c.precision, c.radius_mode, c.k_max, c.k_side = dim, precision, radius_mode, k_max, k_side
    c.k_per_side, c.limiter, c.estimator = k_per_side, limiter, estimator
    c.gamma, c.radius, c.kappa, c.flat_eps, c.active_frac = gamma, radius, kappa, flat_eps, active_frac
    for k in range(5):
        c.s_ref[k] = float(s_ref[k]) if k < len(s_ref) else 0.0
    c.tau32, c.tau64, c.max_level = tau32, tau64, max_level
    for k in range(3):
        c.periodic[k] = int(periodic[k])
        c.box_lo[k] = float(box_lo[k])
        c.box_hi[k] = float(box_hi[k])
    c.n_fluid, c.capacity = int(n_fluid), int(capacity)
    c.mlp_tau_lo, c.mlp_audit, c.max_sims = float(mlp_tau_lo), int(mlp_audit), int(max_sims)
    c.refine, c.refine_ratio = int(refine), float(refine_ratio)
    return c


@dataclass
class ParticleSet:
    """Device SoA particle arrays (torch.cuda tensors) owned by the caller."""
    x: list
    V: object
    u: list
    P: object
    m: object
    id: object
    count: object = None      # particles in use when the arrays hold more room (None: all)

    @property
    def n(self):
        return int(self.V.shape[0]) if self.count is None else int(self.count)

    @property
    def capacity(self):
        return int(self.V.shape[0])

    @staticmethod
    def with_capacity(state, capacity, device="cuda"):
        """Device arrays of `capacity` particles holding `state` in their first n."""
        import torch
        n = state["V"].shape[0]
        assert capacity >= n

        def t(a, dt=torch.float64):
            v = torch.zeros(capacity, dtype=dt, device=device)
            v[:n] = torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=device)
            return v
        return ParticleSet([t(a) for a in state["x"]], t(state["V"]), [t(a) for a in state["u"]], t(state["P"]),
                           t(state["m"]), t(state["id"].astype(np.int32), torch.int32), count=n)

    def grown(self, capacity):
        """A copy with room for `capacity` particles (the first n copied)."""
        import torch
        n = self.n

        def g(v):
            w = torch.zeros(capacity, dtype=v.dtype, device=v.device)
            w[:n] = v[:n]
            return w
        return ParticleSet([g(a) for a in self.x], g(self.V), [g(a) for a in self.u], g(self.P), g(self.m),
                           g(self.id), count=n)

    @property
    def dim(self):
        return len(self.x)

    @staticmethod
    def from_state(state, device="cuda"):
        import torch
        t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=device)
        return ParticleSet([t(a) for a in state["x"]], t(state["V"]), [t(a) for a in state["u"]], t(state["P"]),
                           t(state["m"]), t(state["id"].astype(np.int32), torch.int32))

    @staticmethod
    def from_state_host(state, pinned=True):
        """Host (CPU) copies of a state, page-locked unless pinned=False, for
        Context.step_host."""
        import torch
        def t(a, dt=torch.float64):
            v = torch.from_numpy(np.array(a, dtype=np.float64 if dt == torch.float64 else np.int32, copy=True))
            return v.pin_memory() if pinned else v
        return ParticleSet([t(a) for a in state["x"]], t(state["V"]), [t(a) for a in state["u"]], t(state["P"]),
                           t(state["m"]), t(state["id"].astype(np.int32), torch.int32))

    def to_state(self, n_fluid=None):
        n = self.n
        g = lambda a: a[:n].detach().cpu().numpy()
        st = {"x": [g(a) for a in self.x], "V": g(self.V), "u": [g(a) for a in self.u], "P": g(self.P),
              "m": g(self.m), "id": g(self.id).astype(np.uint32)}
        if n_fluid is not None:
            st["n_fluid"] = n_fluid
        return st

    def struct(self) -> Particles:
        p = Particles()
        p.n = self.n
        for k in range(3):
            p.x[k] = self.x[k].data_ptr() if k < self.dim else None
            p.u[k] = self.u[k].data_ptr() if k < self.dim else None
        p.V, p.P, p.m, p.id = self.V.data_ptr(), self.P.data_ptr(), self.m.data_ptr(), self.id.data_ptr()
        return p


def mlp_init_params(seed):
    """He-initialised parameters (W1, b1 = 0, w2, b2 = 0) from a seeded generator."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W1 = rng.normal(0.0, np.sqrt(2.0 / MLP_IN), size=(MLP_H, MLP_IN))
    w2 = rng.normal(0.0, np.sqrt(1.0 / MLP_H), size=MLP_H)
    return np.concatenate([W1.ravel(), np.zeros(MLP_H), w2, [0.0]]).astype(np.float32)


def sort_keys_noalloc(x, keys_out, perm_out, stream=None):
    """Morton keys and sort order of positions x (list of 1 to 3 contiguous CUDA
    float64 tensors of one length n) into caller buffers keys_out (CUDA int64,
    at least n) and perm_out (CUDA int32, at least n), with the library's fixed
    scratch (no allocation)."""
    import torch
    if not 1 <= len(x) <= 3:
        raise ValueError("sort_keys_noalloc: 1 to 3 position arrays")
    n = int(x[0].shape[0])

    def need(t, dtype, what, length):
        if (not isinstance(t, torch.Tensor) or t.dtype != dtype or not t.is_cuda or not t.is_contiguous()
                or t.dim() != 1 or t.shape[0] < length):
            raise ValueError("sort_keys_noalloc: %s must be a contiguous 1-D CUDA %s tensor of length >= %d"
                             % (what, dtype, length))
    for k, a in enumerate(x):
        need(a, torch.float64, "x[%d]" % k, n)
        if a.shape[0] != n:
            raise ValueError("sort_keys_noalloc: the position arrays differ in length")
    need(keys_out, torch.int64, "keys_out", n)
    need(perm_out, torch.int32, "perm_out", n)
    xs = [_ptr(a) for a in x] + [None] * (3 - len(x))
    _check(lib().lp_sort_keys_noalloc(len(x), n, xs[0], xs[1], xs[2], _ptr(keys_out),
                                      _ptr(perm_out), _stream(stream)), "lp_sort_keys_noalloc")


class Context:
    """An lp_ctx: method configuration plus device scratch for `capacity` particles."""

    def __init__(self, cfg: Config):
        self.cfg = cfg
        h = C.c_void_p()
        _check(lib().lp_create(C.byref(cfg), C.byref(h)), "lp_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().lp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build_neighbors(self, ps: ParticleSet, stream=None) -> Neighbors:
        p = ps.struct()
        nb = Neighbors()
        _check(lib().lp_build_neighbors(self.h, C.byref(p), C.byref(nb), _stream(stream)), "lp_build_neighbors")
        return nb

    def export_neighbors(self, n, stream=None):
        import torch
        k = self.cfg.k_max
        dev = "cuda"
        cnt = torch.empty(n, dtype=torch.int32, device=dev)
        tot = torch.empty(n, dtype=torch.int32, device=dev)
        idx = torch.empty((n, k), dtype=torch.int32, device=dev)
        d2 = torch.empty(n, dtype=torch.float64, device=dev)
        keys = torch.empty(n, dtype=torch.int64, device=dev)
        _check(lib().lp_export_neighbors(self.h, _ptr(cnt), _ptr(tot), _ptr(idx), _ptr(d2), _ptr(keys),
                                         _stream(stream)), "lp_export_neighbors")
        return cnt, tot, idx, d2, keys

    def grid_info(self, stream=None):
        out = (C.c_double * 5)()
        _check(lib().lp_grid_info(self.h, out, _stream(stream)), "lp_grid_info")
        return list(out)

    def gfd_derivs(self, ps: ParticleSet, fields, out_dtype=OUT_F64, status=None, stream=None):
        import torch
        nu = {1: 2, 2: 5, 3: 9}[ps.dim]
        out = torch.empty((len(fields), ps.n, nu), dtype=torch.float64 if out_dtype == OUT_F64 else torch.float32,
                          device="cuda")
        ptrs = (C.c_void_p * len(fields))(*[f.data_ptr() for f in fields])
        p = ps.struct()
        _check(lib().lp_gfd_derivs(self.h, C.byref(p), ptrs, len(fields), out_dtype, _ptr(out), _ptr(status),
                                   _stream(stream)), "lp_gfd_derivs")
        return out

    def onesided_derivs(self, ps: ParticleSet, fields, stream=None):
        import torch
        out = torch.empty((ps.n, ps.dim, 2, len(fields)), dtype=torch.float64, device="cuda")
        ptrs = (C.c_void_p * len(fields))(*[f.data_ptr() for f in fields])
        p = ps.struct()
        _check(lib().lp_onesided_derivs(self.h, C.byref(p), ptrs, len(fields), _ptr(out), _stream(stream)),
               "lp_onesided_derivs")
        return out

    def step(self, ps: ParticleSet, dt=0.0, cfl=0.4, t=None, flag=None, phi=None, r=None, features=None,
             gate_p=None, stream=None):
        p = ps.struct()
        d = _diag(flag, phi, r, features, gate_p)
        _check(lib().lp_step(self.h, C.byref(p), float(dt), float(cfl), _ptr(t), C.byref(d), _stream(stream)),
               "lp_step")

    def step_host(self, ps: ParticleSet, dt=0.0, cfl=0.4, t=None, flag=None, phi=None, r=None, features=None,
                  gate_p=None, stream=None):
        """lp_step on a ParticleSet of host (CPU, ideally pinned) tensors; t and the
        diagnostics are device tensors as for step."""
        p = ps.struct()
        d = _diag(flag, phi, r, features, gate_p)
        _check(lib().lp_step_host(self.h, C.byref(p), float(dt), float(cfl), _ptr(t), C.byref(d), _stream(stream)),
               "lp_step_host")

    def step_batched(self, ps: ParticleSet, offsets, nsim, dt=0.0, cfl=0.4, t=None, flag=None, phi=None, r=None,
                     features=None, gate_p=None, stream=None):
        """One step of nsim simulations stored back to back; offsets: device int64 [nsim + 1]."""
        p = ps.struct()
        d = _diag(flag, phi, r, features, gate_p)
        _check(lib().lp_step_batched(self.h, C.byref(p), _ptr(offsets), int(nsim), float(dt), float(cfl), _ptr(t),
                                     C.byref(d), _stream(stream)), "lp_step_batched")

    def graph_capture(self, ps: ParticleSet, offsets=None, nsim=1, dt=0.0, cfl=0.4, t=None, stream=None):
        """Capture one (batched) step into a CUDA graph on `stream` (a created stream)."""
        self._graph_ps = ps.struct()      # the captured addresses must stay alive
        _check(lib().lp_graph_capture(self.h, C.byref(self._graph_ps), _ptr(offsets), int(nsim), float(dt),
                                      float(cfl), _ptr(t), _stream(stream)), "lp_graph_capture")

    def graph_launch(self, stream=None):
        _check(lib().lp_graph_launch(self.h, _stream(stream)), "lp_graph_launch")

    def set_schedule(self, schedule: int):
        _check(lib().lp_set_schedule(self.h, int(schedule)), "lp_set_schedule")

    def schedule(self) -> int:
        v = C.c_int32()
        _check(lib().lp_get_schedule(self.h, C.byref(v)), "lp_get_schedule")
        return v.value

    def autotune(self, ps: ParticleSet, offsets=None, nsim=1, dt=0.0, cfl=0.4, reps=3, stream=None):
        """Time the query and the fit pass under each schedule on this state and
        keep the faster of each; returns {fit_fused, fit_split, query_tile,
        query_warp, query_tile_queue, fit_split_queue} in ms (0: not offered).
        The state is not changed."""
        p = ps.struct()
        out = (C.c_double * AUTOTUNE_TIMES)()
        _check(lib().lp_autotune(self.h, C.byref(p), _ptr(offsets), int(nsim), float(dt), float(cfl), int(reps),
                                 out, _stream(stream)), "lp_autotune")
        return {"fit_fused": out[0], "fit_split": out[1], "query_tile": out[2], "query_warp": out[3],
                "query_tile_queue": out[4], "fit_split_queue": out[5]}

    def stats(self, stream=None) -> dict:
        s = Stats()
        _check(lib().lp_get_stats(self.h, C.byref(s), _stream(stream)), "lp_get_stats")
        return s.as_dict()

    def reset_stats(self, stream=None):
        _check(lib().lp_reset_stats(self.h, _stream(stream)), "lp_reset_stats")

    # ---- learned estimator -------------------------------------------------
    def mlp_set_params(self, params):
        a = np.ascontiguousarray(params, dtype=np.float32)
        assert a.size == MLP_NPARAM
        _check(lib().lp_mlp_set_params(self.h, a.ctypes.data_as(C.c_void_p)), "lp_mlp_set_params")

    def mlp_get_params(self):
        """(FP32 master weights, BF16 weights as float32) on the host."""
        m = np.zeros(MLP_NPARAM, np.float32)
        b = np.zeros(MLP_NPARAM, np.float32)
        _check(lib().lp_mlp_get_params(self.h, m.ctypes.data_as(C.c_void_p), b.ctypes.data_as(C.c_void_p)),
               "lp_mlp_get_params")
        return m, b

    def mlp_grad(self, X, y, pos_weight, stream=None):
        import torch
        g = torch.empty(MLP_NPARAM, dtype=torch.float32, device="cuda")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        _check(lib().lp_mlp_grad(self.h, _ptr(X), _ptr(y), int(X.shape[0]), float(pos_weight), _ptr(g), _ptr(loss),
                                 _stream(stream)), "lp_mlp_grad")
        return g, loss

    def mlp_adam_step(self, grad, lr, stream=None):
        _check(lib().lp_mlp_adam_step(self.h, _ptr(grad), float(lr), _stream(stream)), "lp_mlp_adam_step")

    def mlp_train(self, X, y, epochs, batch, lr, pos_weight, stream=None):
        losses = np.zeros(epochs, np.float32)
        _check(lib().lp_mlp_train(self.h, _ptr(X), _ptr(y), int(X.shape[0]), int(epochs), int(batch), float(lr),
                                  float(pos_weight), losses.ctypes.data_as(C.c_void_p), _stream(stream)),
               "lp_mlp_train")
        return losses

    def mlp_infer(self, X, stream=None):
        import torch
        p = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
        _check(lib().lp_mlp_infer(self.h, _ptr(X), int(X.shape[0]), _ptr(p), _stream(stream)), "lp_mlp_infer")
        return p

    def set_profiling(self, on=True):
        _check(lib().lp_set_profiling(self.h, 1 if on else 0), "lp_set_profiling")

    def phase_times(self, stream=None):
        """{phase name: (milliseconds, launches)} since the last call."""
        ms = (C.c_double * NPHASES)()
        nl = (C.c_int64 * NPHASES)()
        _check(lib().lp_phase_times(self.h, ms, nl, _stream(stream)), "lp_phase_times")
        return {lib().lp_phase_name(k).decode(): (ms[k], nl[k]) for k in range(NPHASES)}

    def dt_device_ptr(self):
        return lib().lp_dt_device(self.h)

    # ---- reservoir inflow and capacity ---------------------------------------
    def inflow(self, ps: ParticleSet, inlet: Inlet, stream=None):
        """Reservoir inflow through `inlet` (lp_inflow): appends the particles
        that entered into the room of ps (ps.count grows); returns the inflow
        state of the call.  LPError(ERR_CAPACITY) when ps has no room."""
        p = ps.struct()
        n_out = C.c_int64(0)
        info = InflowInfo()
        _check(lib().lp_inflow(self.h, C.byref(p), ps.capacity, C.byref(inlet), C.byref(n_out), C.byref(info),
                               _stream(stream)), "lp_inflow")
        ps.count = int(n_out.value)
        return info.as_dict()

    def remove_outside(self, ps: ParticleSet, lo, hi, stream=None):
        """Outflow: drop the particles outside the box [lo, hi] (lp_remove_outside);
        ps.count shrinks.  Returns the number removed."""
        p = ps.struct()
        n_out = C.c_int64(0)
        lo_a = (C.c_double * 3)(*[float(v) for v in lo])
        hi_a = (C.c_double * 3)(*[float(v) for v in hi])
        _check(lib().lp_remove_outside(self.h, C.byref(p), lo_a, hi_a, C.byref(n_out), _stream(stream)),
               "lp_remove_outside")
        removed = ps.n - int(n_out.value)
        ps.count = int(n_out.value)
        return removed

    def free_surface_ghosts(self, ps: ParticleSet, min_per_side=1, p_ghost=0.0, ghost_base=2 ** 31, stream=None):
        """Free-surface ghosts (lp_free_surface_ghosts): builds the lists (ps is
        permuted into key order) and appends a ghost for each incomplete axis
        direction of each fluid particle into the room of ps (ps.count grows).
        Returns the number appended.  LPError(ERR_CAPACITY) when ps has no room."""
        p = ps.struct()
        n_out = C.c_int64(0)
        _check(lib().lp_free_surface_ghosts(self.h, C.byref(p), ps.capacity, int(min_per_side), float(p_ghost),
                                            int(ghost_base), C.byref(n_out), _stream(stream)),
               "lp_free_surface_ghosts")
        added = int(n_out.value) - ps.n
        ps.count = int(n_out.value)
        return added

    def remove_ghosts(self, ps: ParticleSet, first_id=2 ** 31, stream=None):
        """Drop the particles with id >= first_id (lp_remove_ghosts); returns the
        number removed."""
        p = ps.struct()
        n_out = C.c_int64(0)
        _check(lib().lp_remove_ghosts(self.h, C.byref(p), int(first_id), C.byref(n_out), _stream(stream)),
               "lp_remove_ghosts")
        removed = ps.n - int(n_out.value)
        ps.count = int(n_out.value)
        return removed

    def octant_coverage(self, gap=None, stream=None):
        """All-octant coverage of the last build's lists (lp_octant_coverage):
        the number of particles whose list misses an octant; gap (device uint8
        tensor of n, optional) receives the per-particle flags in key order."""
        n_gap = C.c_int64(0)
        _check(lib().lp_octant_coverage(self.h, _ptr(gap), C.byref(n_gap), _stream(stream)), "lp_octant_coverage")
        return int(n_gap.value)

    def reserve(self, capacity):
        """Resize the context's scratch to `capacity` particles (lp_reserve)."""
        _check(lib().lp_reserve(self.h, int(capacity)), "lp_reserve")
        self.cfg.capacity = int(capacity)
