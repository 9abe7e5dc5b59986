"""Python binding of the C ABI in ``include/cch.h`` (argument marshalling only).

Every step of the collision-handling path runs inside ``libcch.so``; this
module converts torch tensors and numpy arrays into the plain pointers and
sizes the C ABI takes.  Position tensors must be contiguous float64 CUDA
tensors of shape (n_verts, 3).  There is no CPU fallback: if the library
cannot be loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional, Sequence

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

CCH_OK = 0
STATUS = {0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "HBM budget exceeded", 4: "CUDA error",
          5: "internal capacity exceeded", 6: "bounded device loop timed out", 7: "input state intersects",
          8: "cancelled", 9: "invalid state"}


class CchError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)} ({code})")
        self.code = code


class Params(C.Structure):
    _fields_ = [("d_min", C.c_double), ("d_max", C.c_double), ("delta", C.c_double), ("sigma", C.c_double),
                ("gamma", C.c_double), ("eps", C.c_double), ("jacobi_omega", C.c_double),
                ("max_iters", C.c_int32), ("gs_sweeps", C.c_int32), ("precision", C.c_int32),
                ("solver", C.c_int32), ("ccd_check", C.c_int32), ("accept_check", C.c_int32),
                ("validate_input", C.c_int32), ("iters_per_launch", C.c_int32), ("bvh_refit_only", C.c_int32),
                ("constraint_form", C.c_int32), ("step_rule", C.c_int32), ("ccd_rounds", C.c_int32),
                ("seed", C.c_uint64), ("max_polls", C.c_int32), ("pair_capacity", C.c_int32),
                ("sweep_blocks", C.c_int32), ("colouring", C.c_int32)]


class Topology(C.Structure):
    _fields_ = [("n_verts", C.c_int64), ("inv_mass", C.c_void_p), ("point_radius", C.c_void_p),
                ("n_tris", C.c_int64), ("tris", C.c_void_p), ("n_edges", C.c_int64), ("edges", C.c_void_p),
                ("n_len", C.c_int64), ("len_edges", C.c_void_p), ("n_points", C.c_int64), ("points", C.c_void_p)]


class StepStats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("searches", C.c_int32), ("converged", C.c_int32),
                ("ccd_clamps", C.c_int32), ("pairs_evaluated", C.c_int64), ("max_pairs", C.c_int64),
                ("active_contacts", C.c_int64), ("candidates", C.c_int64), ("degenerate", C.c_int64),
                ("max_vertex_contacts", C.c_int32), ("max_vertex_edges", C.c_int32), ("final_r_inf", C.c_double),
                ("min_pair_dist", C.c_double), ("intersections", C.c_int64), ("uncertain", C.c_int64),
                ("device_ms", C.c_double), ("kernel_launches", C.c_int64), ("gs_depth", C.c_int32),
                ("frozen_vertices", C.c_int32), ("contact_vertices", C.c_int64), ("contact_colours", C.c_int32),
                ("edge_colours", C.c_int32), ("pair_vertices", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TuneResult(C.Structure):
    _fields_ = [("iters_per_launch", C.c_int32), ("query_block", C.c_int32), ("bvh_refit_only", C.c_int32),
                ("trials", C.c_int32), ("consistent", C.c_int32), ("packet_traversal", C.c_int32),
                ("best_ms", C.c_double), ("default_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libcch.so (building it in-tree when the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not _build.up_to_date():
                try:
                    path = _build.build()
                except Exception as e:  # no silent fallback: the CUDA path is the product
                    raise RuntimeError(f"libcch.so is missing and could not be built: {e}") from e
            L = C.CDLL(path)
            p, i32, i64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
            L.cch_params_default.argtypes = [C.POINTER(Params)]
            L.cch_status_string.restype = C.c_char_p
            L.cch_status_string.argtypes = [C.c_int]
            L.cch_create_scene.argtypes = [C.POINTER(Topology), C.POINTER(Params), p, C.POINTER(p)]
            L.cch_create_batch.argtypes = [C.POINTER(Topology), i32, C.POINTER(Params), p, C.POINTER(p)]
            L.cch_create_batch_params.argtypes = [C.POINTER(Topology), i32, C.POINTER(Params), C.POINTER(Params), p,
                                                  C.POINTER(p)]
            L.cch_handle_step.argtypes = [p, p, p, p, C.POINTER(StepStats)]
            L.cch_handle_step_host.argtypes = [p, p, p, p, C.POINTER(StepStats)]
            L.cch_batch_handle_step.argtypes = [p, C.POINTER(p), C.POINTER(p), C.POINTER(p), C.POINTER(StepStats)]
            L.cch_destroy.argtypes = [p]
            L.cch_query_pairs.argtypes = [p, p, p, d, i32, p, p, i64, C.POINTER(i64)]
            L.cch_server_create.argtypes = [C.c_size_t, C.POINTER(Params), i32, p, C.POINTER(p)]
            L.cch_server_add_scene.argtypes = [p, C.POINTER(Topology), C.POINTER(i32)]
            L.cch_server_add_scene_params.argtypes = [p, C.POINTER(Topology), C.POINTER(Params), C.POINTER(i32)]
            L.cch_server_submit.argtypes = [p, i32, p, p, p, C.POINTER(C.c_uint64)]
            L.cch_server_wait.argtypes = [p, C.c_uint64, C.POINTER(StepStats), C.POINTER(d)]
            L.cch_server_destroy.argtypes = [p]
            L.cch_query_pairs_noalloc.argtypes = [p, p, p, d, i32, p, p, i64, C.POINTER(i64)]
            L.cch_set_profiling.argtypes = [p, i32]
            L.cch_get_profile.argtypes = [p, p, p, i32]
            L.cch_autotune.argtypes = [p, p, p, i32, C.POINTER(TuneResult)]
            L.cch_set_max_polls.argtypes = [p, i32]
            L.cch_normal_flow_target.argtypes = [p, p, d, d, d, i32, p]
            L.cch_friction_filter.argtypes = [p, p, p, p, d, d, d]
            for f in ("cch_params_default", "cch_create_scene", "cch_create_batch", "cch_create_batch_params",
                      "cch_server_add_scene_params", "cch_handle_step",
                      "cch_handle_step_host", "cch_batch_handle_step", "cch_destroy", "cch_query_pairs",
                      "cch_server_create", "cch_server_add_scene", "cch_server_submit", "cch_server_wait",
                      "cch_server_destroy", "cch_set_profiling", "cch_get_profile", "cch_query_pairs_noalloc",
                      "cch_autotune", "cch_set_max_polls", "cch_normal_flow_target", "cch_friction_filter"):
                getattr(L, f).restype = C.c_int
            _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != CCH_OK:
        raise CchError(rc, what)


def params(**kw) -> Params:
    p = Params()
    _check(lib().cch_params_default(C.byref(p)), "cch_params_default")
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def params_for(scene, **kw) -> Params:
    d = dict(getattr(scene, "params", {}) or {})
    d.update(kw)
    return params(**d)


class _Topo:
    """Contiguous host copies of one scene's topology and its ctypes view."""

    def __init__(self, scene):
        self.n = int(scene.n_verts)
        self.inv_mass = np.ascontiguousarray(scene.inv_mass, dtype=np.float64)
        r = getattr(scene, "radius", None)
        self.radius = None if r is None else np.ascontiguousarray(r, dtype=np.float64)
        self.tris = np.ascontiguousarray(scene.tris, dtype=np.int32).reshape(-1, 3)
        self.edges = np.ascontiguousarray(scene.edges, dtype=np.int32).reshape(-1, 2)
        self.len_edges = np.ascontiguousarray(scene.len_edges, dtype=np.int32).reshape(-1, 2)
        self.points = np.ascontiguousarray(scene.points, dtype=np.int32).reshape(-1)

        def ptr(a):
            return None if a is None or a.size == 0 else a.ctypes.data

        self.c = Topology(self.n, ptr(self.inv_mass), ptr(self.radius), len(self.tris), ptr(self.tris),
                          len(self.edges), ptr(self.edges), len(self.len_edges), ptr(self.len_edges),
                          len(self.points), ptr(self.points))


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(stream)


def _dev_ptr(t, n):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("positions must be contiguous float64 CUDA tensors")
    if tuple(t.shape) != (n, 3):
        raise ValueError(f"positions must have shape ({n}, 3), got {tuple(t.shape)}")
    return t.data_ptr()


class Scene:
    """A resident scene (or a batch of scenes) on the current CUDA device."""

    def __init__(self, scenes, prm: Optional[Params] = None, stream=None, scene_params=None):
        """scene_params: optional per-scene Params whose physical fields (d_min,
        d_max, delta, sigma, gamma, eps, max_iters, seed) replace prm's for
        that scene (cch_create_batch_params)."""
        single = not isinstance(scenes, (list, tuple))
        self.single = single
        self._scenes = [scenes] if single else list(scenes)
        self.topos = [_Topo(s) for s in self._scenes]
        self.prm = prm if prm is not None else params_for(self._scenes[0])
        self.stream = _stream_ptr(stream)
        arr = (Topology * len(self.topos))(*[t.c for t in self.topos])
        h = C.c_void_p()
        if scene_params is None:
            _check(lib().cch_create_batch(arr, len(self.topos), C.byref(self.prm), C.c_void_p(self.stream),
                                          C.byref(h)), "cch_create_batch")
        else:
            if len(scene_params) != len(self.topos):
                raise ValueError("one Params per scene")
            sp = (Params * len(self.topos))(*scene_params)
            _check(lib().cch_create_batch_params(arr, len(self.topos), C.byref(self.prm), sp,
                                                 C.c_void_p(self.stream), C.byref(h)), "cch_create_batch_params")
        self.h = h

    @property
    def n_verts(self):
        return self.topos[0].n

    def step(self, x_t, x_tilde, out=None):
        """One Algorithm 1 call on device tensors; returns (x_next, stats)."""
        import torch
        if not self.single:
            raise ValueError("use batch_step for a batch")
        n = self.topos[0].n
        if out is None:
            out = torch.empty_like(x_t)
        st = StepStats()
        _check(lib().cch_handle_step(self.h, C.c_void_p(_dev_ptr(x_t, n)), C.c_void_p(_dev_ptr(x_tilde, n)),
                                     C.c_void_p(_dev_ptr(out, n)), C.byref(st)), "cch_handle_step")
        return out, st.as_dict()

    def step_host(self, x_t: np.ndarray, x_tilde: np.ndarray, out: Optional[np.ndarray] = None):
        """The same call with host (numpy) buffers; copies happen in the library."""
        n = self.topos[0].n
        a = np.ascontiguousarray(x_t, dtype=np.float64).reshape(n, 3)
        b = np.ascontiguousarray(x_tilde, dtype=np.float64).reshape(n, 3)
        if out is None:
            out = np.empty((n, 3))
        st = StepStats()
        _check(lib().cch_handle_step_host(self.h, C.c_void_p(a.ctypes.data), C.c_void_p(b.ctypes.data),
                                          C.c_void_p(out.ctypes.data), C.byref(st)), "cch_handle_step_host")
        return out, st.as_dict()

    def batch_step(self, xs_t: Sequence, xs_tilde: Sequence, outs: Optional[Sequence] = None):
        import torch
        k = len(self.topos)
        if outs is None:
            outs = [torch.empty_like(x) for x in xs_t]
        P = C.c_void_p * k
        a = P(*[_dev_ptr(x, t.n) for x, t in zip(xs_t, self.topos)])
        b = P(*[_dev_ptr(x, t.n) for x, t in zip(xs_tilde, self.topos)])
        o = P(*[_dev_ptr(x, t.n) for x, t in zip(outs, self.topos)])
        st = (StepStats * k)()
        _check(lib().cch_batch_handle_step(self.h, a, b, o, st), "cch_batch_handle_step")
        return outs, [s.as_dict() for s in st]

    def query_pairs(self, x, x_ref, D: float, candidates: bool = False, step_search: bool = False):
        """Candidate set (candidates=True), proximity set P at bound D with
        exact distances, or (step_search=True) P as the first search of a
        step forms it at the scene's D^max, with the distances it records."""
        n = self.topos[0].n
        mode = 2 if step_search else int(bool(candidates))
        cnt = C.c_int64(0)
        _check(lib().cch_query_pairs(self.h, C.c_void_p(_dev_ptr(x, n)), C.c_void_p(_dev_ptr(x_ref, n)), float(D),
                                     mode, None, None, 0, C.byref(cnt)), "cch_query_pairs")
        m = cnt.value
        keys = np.zeros(max(m, 1), np.uint64)
        dist = np.zeros(max(m, 1), np.float64)
        _check(lib().cch_query_pairs(self.h, C.c_void_p(_dev_ptr(x, n)), C.c_void_p(_dev_ptr(x_ref, n)), float(D),
                                     mode, C.c_void_p(keys.ctypes.data),
                                     C.c_void_p(dist.ctypes.data), m, C.byref(cnt)), "cch_query_pairs")
        o = np.argsort(keys[:m], kind="stable")
        return keys[:m][o], dist[:m][o]

    NOALLOC_MAX_PAIRS = 131072

    def query_pairs_noalloc(self, x, x_ref, D: float, candidates: bool, cap: int = NOALLOC_MAX_PAIRS):
        """The allocation-free variant of query_pairs (fixed library-side scratch).

        Returns (keys, dist) sorted by key; raises CchError with code 5
        (internal capacity exceeded) when more than NOALLOC_MAX_PAIRS pairs
        are found."""
        n = self.topos[0].n
        keys = np.zeros(max(cap, 1), np.uint64)
        dist = np.zeros(max(cap, 1), np.float64)
        cnt = C.c_int64(0)
        _check(lib().cch_query_pairs_noalloc(self.h, C.c_void_p(_dev_ptr(x, n)), C.c_void_p(_dev_ptr(x_ref, n)),
                                             float(D), int(bool(candidates)), C.c_void_p(keys.ctypes.data),
                                             C.c_void_p(dist.ctypes.data), cap, C.byref(cnt)),
               "cch_query_pairs_noalloc")
        m = min(cnt.value, cap)
        o = np.argsort(keys[:m], kind="stable")
        return keys[:m][o], dist[:m][o]

    def normal_flow_target(self, x, beta: float, alpha: float, sign: float, iters: int = 3, out=None):
        """Target of the normal flow of Sec. 7.4 at x (device tensors)."""
        import torch
        n = self.topos[0].n
        if out is None:
            out = torch.empty_like(x)
        _check(lib().cch_normal_flow_target(self.h, C.c_void_p(_dev_ptr(x, n)), float(beta), float(alpha),
                                            float(sign), int(iters), C.c_void_p(_dev_ptr(out, n))),
               "cch_normal_flow_target")
        return out

    def friction_filter(self, x, y, mu: float, reach: float, sep: float, out=None):
        """Velocity filter of Sec. 6.3 on the frictionless target y (device tensors)."""
        import torch
        n = self.topos[0].n
        if out is None:
            out = torch.empty_like(y)
        _check(lib().cch_friction_filter(self.h, C.c_void_p(_dev_ptr(x, n)), C.c_void_p(_dev_ptr(y, n)),
                                         C.c_void_p(_dev_ptr(out, n)), float(mu), float(reach), float(sep)),
               "cch_friction_filter")
        return out

    def set_max_polls(self, max_polls: int):
        """Bound of the scene's bounded device waits (0 = the default)."""
        _check(lib().cch_set_max_polls(self.h, int(max_polls)), "cch_set_max_polls")

    def autotune(self, x_t, x_tilde, probe_iters: int = 64):
        """Times launch configurations on a probe step from (x_t, x_tilde) and
        keeps the fastest for later steps; returns the choice and timings."""
        n = self.topos[0].n
        r = TuneResult()
        _check(lib().cch_autotune(self.h, C.c_void_p(_dev_ptr(x_t, n)), C.c_void_p(_dev_ptr(x_tilde, n)),
                                  int(probe_iters), C.byref(r)), "cch_autotune")
        return r.as_dict()

    PROFILE_GROUPS = ("refit", "query_vt", "query_ee", "query_vv", "refresh", "assemble", "order", "sweep",
                      "forward", "control", "setup", "output", "finalize", "colour")

    def set_profiling(self, on: bool):
        _check(lib().cch_set_profiling(self.h, int(bool(on))), "cch_set_profiling")

    def profile(self):
        n = len(self.PROFILE_GROUPS)
        ms = np.zeros(n)
        cnt = np.zeros(n, np.int64)
        _check(lib().cch_get_profile(self.h, C.c_void_p(ms.ctypes.data), C.c_void_p(cnt.ctypes.data), n),
               "cch_get_profile")
        return {g: (float(ms[i]), int(cnt[i])) for i, g in enumerate(self.PROFILE_GROUPS)}

    def close(self):
        if getattr(self, "h", None):
            lib().cch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Resident scenes plus a request loop with continuous batching (C ABI
    cch_server_*).  Requests take device tensors that must stay alive until
    wait() returns."""

    def __init__(self, hbm_budget_bytes: int, prm: Optional[Params] = None, max_active: int = 8, stream=None):
        self.prm = prm if prm is not None else params()
        self.stream = _stream_ptr(stream)
        h = C.c_void_p()
        _check(lib().cch_server_create(C.c_size_t(int(hbm_budget_bytes)), C.byref(self.prm), int(max_active),
                                       C.c_void_p(self.stream), C.byref(h)), "cch_server_create")
        self.h = h
        self.n = []
        self._keep = {}

    def add_scene(self, scene, prm: Optional[Params] = None) -> int:
        """Make a scene resident; prm: its own physical parameters (see
        Scene's scene_params), else the server's."""
        t = _Topo(scene)
        sid = C.c_int32(-1)
        if prm is None:
            _check(lib().cch_server_add_scene(self.h, C.byref(t.c), C.byref(sid)), "cch_server_add_scene")
        else:
            _check(lib().cch_server_add_scene_params(self.h, C.byref(t.c), C.byref(prm), C.byref(sid)),
                   "cch_server_add_scene_params")
        self.n.append(t.n)
        return sid.value

    def submit(self, scene_id: int, x_t, x_tilde, out) -> int:
        n = self.n[scene_id]
        tk = C.c_uint64(0)
        _check(lib().cch_server_submit(self.h, int(scene_id), C.c_void_p(_dev_ptr(x_t, n)),
                                       C.c_void_p(_dev_ptr(x_tilde, n)), C.c_void_p(_dev_ptr(out, n)), C.byref(tk)),
               "cch_server_submit")
        self._keep[tk.value] = (x_t, x_tilde, out)
        return tk.value

    def wait(self, ticket: int):
        st = StepStats()
        lat = C.c_double(0.0)
        rc = lib().cch_server_wait(self.h, C.c_uint64(ticket), C.byref(st), C.byref(lat))
        self._keep.pop(ticket, None)
        _check(rc, "cch_server_wait")
        return st.as_dict(), lat.value

    def close(self):
        if getattr(self, "h", None):
            lib().cch_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
