"""CPU FP64 oracle of the two-way collision-handling step (arXiv 2211.04045).

TEST INFRASTRUCTURE ONLY.  This package wraps ``cch_oracle.c``, the plain,
slow reference that the CUDA path is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it; the product package never does.  It shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cch_oracle.c")
_HDR = os.path.join(_HERE, "cch_oracle.h")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

VT, EE, VV = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FP contraction, IEEE semantics)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < newest:
        tmp = _OUT + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-Wall", "-Wno-unused-function", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OUT)
    return _OUT


class Topology(C.Structure):
    _fields_ = [("n_verts", C.c_int64), ("inv_mass", C.c_void_p), ("radius", C.c_void_p),
                ("n_tris", C.c_int64), ("tris", C.c_void_p), ("n_edges", C.c_int64), ("edges", C.c_void_p),
                ("n_len", C.c_int64), ("len_edges", C.c_void_p), ("n_points", C.c_int64), ("points", C.c_void_p)]


class Params(C.Structure):
    _fields_ = [("d_min", C.c_double), ("d_max", C.c_double), ("delta", C.c_double), ("sigma", C.c_double),
                ("gamma", C.c_double), ("eps", C.c_double), ("jacobi_omega", C.c_double),
                ("max_iters", C.c_int32), ("gs_sweeps", C.c_int32), ("solver", C.c_int32),
                ("ccd_check", C.c_int32), ("search_mode", C.c_int32), ("constraint_form", C.c_int32),
                ("step_rule", C.c_int32), ("ccd_rounds", C.c_int32), ("colouring", C.c_int32),
                ("seed", C.c_uint64)]


class Stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("searches", C.c_int32), ("converged", C.c_int32),
                ("ccd_clamps", C.c_int32), ("pairs_evaluated", C.c_int64), ("max_pairs", C.c_int64),
                ("active_contacts", C.c_int64), ("candidates", C.c_int64), ("degenerate", C.c_int64),
                ("max_vertex_contacts", C.c_int32), ("max_vertex_edges", C.c_int32), ("final_r_inf", C.c_double),
                ("min_pair_dist", C.c_double), ("frozen_vertices", C.c_int32), ("contact_colours", C.c_int32),
                ("contact_vertices", C.c_int64), ("edge_colours", C.c_int32), ("reserved_", C.c_int32),
                ("pair_vertices", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Trace(C.Structure):
    _fields_ = [("cap_iters", C.c_int32), ("x", C.c_void_p), ("y", C.c_void_p), ("Dl", C.c_void_p),
                ("Di", C.c_void_p), ("searched", C.c_void_p), ("n_pairs", C.c_void_p), ("cap_pairs", C.c_int64),
                ("pair_keys", C.c_void_p), ("n_contacts", C.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            d, p, i64, i32, u64 = C.c_double, C.c_void_p, C.c_int64, C.c_int32, C.c_uint64
            L.orc_params_default.argtypes = [C.POINTER(Params)]
            L.orc_point_segment_dist.restype = d
            L.orc_point_segment_dist.argtypes = [p, p, p, p]
            L.orc_point_triangle_dist.restype = d
            L.orc_point_triangle_dist.argtypes = [p, p, p, p]
            L.orc_segment_segment_dist.restype = d
            L.orc_segment_segment_dist.argtypes = [p, p, p, p, p, p]
            L.orc_signed_volume.restype = d
            L.orc_signed_volume.argtypes = [p, p, p, p]
            L.orc_orient3d_exact.restype = C.c_int
            L.orc_orient3d_exact.argtypes = [p, p, p, p]
            L.orc_splitmix64.restype = u64
            L.orc_splitmix64.argtypes = [u64]
            L.orc_candidates.restype = i64
            L.orc_candidates.argtypes = [C.POINTER(Topology), p, p, d, i32, p, i64]
            L.orc_proximity.restype = i64
            L.orc_proximity.argtypes = [C.POINTER(Topology), p, p, d, i32, p, p, i64]
            L.orc_contact_constraint.restype = C.c_int
            L.orc_contact_constraint.argtypes = [C.c_int, p, p, d, C.c_int, p, p]
            L.orc_backward_once.restype = C.c_int
            L.orc_backward_once.argtypes = [C.POINTER(Topology), C.POINTER(Params), p, p, p, p]
            L.orc_colouring.restype = i32
            L.orc_colouring.argtypes = [i32, i64, p, p, p, i64, p]
            L.orc_contact_colours.restype = i64
            L.orc_contact_colours.argtypes = [C.POINTER(Topology), C.POINTER(Params), p, p, p, p, i64]
            L.orc_edge_colours.restype = i32
            L.orc_edge_colours.argtypes = [C.POINTER(Topology), C.POINTER(Params), p]
            L.orc_ccd_conservative.restype = C.c_int
            L.orc_ccd_conservative.argtypes = [C.c_int, p, p, p, d]
            L.orc_ccd.restype = C.c_int
            L.orc_ccd.argtypes = [C.c_int, p, p, p, p]
            L.orc_count_intersections.restype = i64
            L.orc_count_intersections.argtypes = [C.POINTER(Topology), p]
            L.orc_handle_step.restype = C.c_int
            L.orc_handle_step.argtypes = [C.POINTER(Topology), C.POINTER(Params), p, p, p, C.POINTER(Stats),
                                          C.POINTER(Trace)]
            _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a):
    return a.ctypes.data if a is not None and a.size else None


class OracleScene:
    """Holds the contiguous arrays of one scene and the ctypes topology."""

    def __init__(self, scene):
        self.n = int(scene.n_verts)
        self.inv_mass = _f64(scene.inv_mass)
        self.radius = None if scene.radius is None else _f64(scene.radius)
        self.tris = _i32(scene.tris).reshape(-1, 3)
        self.edges = _i32(scene.edges).reshape(-1, 2)
        self.len_edges = _i32(scene.len_edges).reshape(-1, 2)
        self.points = _i32(scene.points).reshape(-1)
        self.topo = Topology(self.n, _ptr(self.inv_mass), None if self.radius is None else _ptr(self.radius),
                             len(self.tris), _ptr(self.tris), len(self.edges), _ptr(self.edges),
                             len(self.len_edges), _ptr(self.len_edges), len(self.points), _ptr(self.points))


def params(**kw) -> Params:
    p = Params()
    lib().orc_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def params_for(scene, **kw) -> Params:
    """Defaults of Table 2 overridden by the scene's own parameters."""
    d = dict(getattr(scene, "params", {}) or {})
    d.update(kw)
    return params(**d)


def handle_step(osc: OracleScene, prm: Params, x_t, x_tilde, trace_iters: int = 0, trace_pairs: int = 0):
    """Algorithm 1 on one step.  Returns (x_next, stats dict, trace dict|None)."""
    x_t = _f64(x_t).reshape(-1, 3)
    x_tilde = _f64(x_tilde).reshape(-1, 3)
    out = np.empty_like(x_t)
    st = Stats()
    tr = None
    bufs = None
    if trace_iters:
        n, ci = osc.n, trace_iters
        bufs = dict(x=np.zeros((ci + 1, n, 3)), y=np.zeros((ci, n, 3)), Dl=np.zeros(ci), Di=np.zeros((ci, n)),
                    searched=np.zeros(ci, np.int32), n_pairs=np.zeros(ci, np.int64),
                    pair_keys=np.zeros((ci, max(trace_pairs, 1)), np.uint64), n_contacts=np.zeros(ci, np.int64))
        tr = Trace(ci, _ptr(bufs["x"]), _ptr(bufs["y"]), _ptr(bufs["Dl"]), _ptr(bufs["Di"]),
                   _ptr(bufs["searched"]), _ptr(bufs["n_pairs"]), max(trace_pairs, 1),
                   _ptr(bufs["pair_keys"]) if trace_pairs else None, _ptr(bufs["n_contacts"]))
    rc = lib().orc_handle_step(C.byref(osc.topo), C.byref(prm), _ptr(x_t), _ptr(x_tilde), _ptr(out), C.byref(st),
                               C.byref(tr) if tr is not None else None)
    if rc != 0:
        raise RuntimeError(f"oracle returned {rc}")
    return out, st.as_dict(), bufs


def candidates(osc: OracleScene, x, D, mode=0, x_tilde=None):
    x = _f64(x).reshape(-1, 3)
    xt = None if x_tilde is None else _f64(x_tilde).reshape(-1, 3)
    L = lib()
    n = L.orc_candidates(C.byref(osc.topo), _ptr(x), _ptr(xt) if xt is not None else None, D, mode, None, 0)
    keys = np.zeros(max(n, 1), np.uint64)
    L.orc_candidates(C.byref(osc.topo), _ptr(x), _ptr(xt) if xt is not None else None, D, mode, _ptr(keys), n)
    return keys[:n]


def proximity(osc: OracleScene, x, D, mode=0, x_tilde=None):
    x = _f64(x).reshape(-1, 3)
    xt = None if x_tilde is None else _f64(x_tilde).reshape(-1, 3)
    L = lib()
    n = L.orc_proximity(C.byref(osc.topo), _ptr(x), _ptr(xt) if xt is not None else None, D, mode, None, None, 0)
    keys = np.zeros(max(n, 1), np.uint64)
    dist = np.zeros(max(n, 1))
    L.orc_proximity(C.byref(osc.topo), _ptr(x), _ptr(xt) if xt is not None else None, D, mode, _ptr(keys),
                    _ptr(dist), n)
    return keys[:n], dist[:n]


def backward_once(osc: OracleScene, prm: Params, x, y_in, y_target):
    x, y_in, y_target = (_f64(a).reshape(-1, 3) for a in (x, y_in, y_target))
    out = np.empty_like(x)
    lib().orc_backward_once(C.byref(osc.topo), C.byref(prm), _ptr(x), _ptr(y_in), _ptr(y_target), _ptr(out))
    return out


def colouring(verts, prio, inv_mass, kind=0):
    """Randomized colouring (Sec. 4.3, R11) of constraints with vertex lists
    verts (m x 4, -1 = absent) and priorities prio: kind 0 greedy, 1 level.
    Returns (colours, count)."""
    verts = np.ascontiguousarray(verts, dtype=np.int32).reshape(-1, 4)
    prio = np.ascontiguousarray(prio, dtype=np.uint64).reshape(-1)
    im = _f64(inv_mass)
    col = np.zeros(max(len(prio), 1), np.int32)
    k = lib().orc_colouring(int(kind), len(prio), _ptr(verts), _ptr(prio), _ptr(im), len(im), _ptr(col))
    return col[:len(prio)], int(k)


def greedy_colouring(verts, prio, inv_mass):
    return colouring(verts, prio, inv_mass, 0)


def contact_colours(osc: OracleScene, prm: Params, x, x_tilde=None):
    """Keys (ascending) and colours of the contact constraints a backward step
    at x builds from a search at D^max."""
    x = _f64(x).reshape(-1, 3)
    xt = x if x_tilde is None else _f64(x_tilde).reshape(-1, 3)
    L = lib()
    n = L.orc_contact_colours(C.byref(osc.topo), C.byref(prm), _ptr(x), _ptr(xt), None, None, 0)
    keys = np.zeros(max(n, 1), np.uint64)
    col = np.zeros(max(n, 1), np.int32)
    L.orc_contact_colours(C.byref(osc.topo), C.byref(prm), _ptr(x), _ptr(xt), _ptr(keys), _ptr(col), n)
    return keys[:n], col[:n]


def edge_colours(osc: OracleScene, prm: Params):
    """Colours of the edge-length constraints, in the topology's edge order."""
    col = np.zeros(max(len(osc.len_edges), 1), np.int32)
    k = lib().orc_edge_colours(C.byref(osc.topo), C.byref(prm), _ptr(col))
    return col[:len(osc.len_edges)], int(k)


def count_intersections(osc: OracleScene, x) -> int:
    x = _f64(x).reshape(-1, 3)
    return int(lib().orc_count_intersections(C.byref(osc.topo), _ptr(x)))


def _v(a):
    return _f64(a).reshape(-1)


def point_segment_dist(p, a, b):
    t = C.c_double()
    arrs = [_v(q) for q in (p, a, b)]
    d = lib().orc_point_segment_dist(*(_ptr(q) for q in arrs), C.addressof(t))
    return d, t.value


def point_triangle_dist(p, a, b, c):
    arrs = [_v(q) for q in (p, a, b, c)]
    return lib().orc_point_triangle_dist(*(_ptr(q) for q in arrs))


def segment_segment_dist(a, b, c, d):
    s, t = C.c_double(), C.c_double()
    arrs = [_v(q) for q in (a, b, c, d)]
    dist = lib().orc_segment_segment_dist(*(_ptr(q) for q in arrs), C.addressof(s), C.addressof(t))
    return dist, s.value, t.value


def signed_volume(a, b, c, d):
    arrs = [_v(q) for q in (a, b, c, d)]
    return lib().orc_signed_volume(*(_ptr(q) for q in arrs))


def orient3d_exact(a, b, c, d):
    arrs = [_v(q) for q in (a, b, c, d)]
    return lib().orc_orient3d_exact(*(_ptr(q) for q in arrs))


def splitmix64(x: int) -> int:
    return int(lib().orc_splitmix64(C.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


def contact_constraint(kind, pos, rho, delta, form=0):
    pos = _f64(pos).reshape(-1)
    rho = _f64(rho).reshape(-1)
    c0 = C.c_double()
    g = np.zeros(12)
    ok = lib().orc_contact_constraint(kind, _ptr(pos), _ptr(rho), delta, int(form), C.addressof(c0), _ptr(g))
    nv = 2 if kind == VV else 4
    return bool(ok), c0.value, g.reshape(4, 3)[:nv]


def ccd(kind, x0, x1, rho=None):
    x0 = _f64(x0).reshape(-1)
    x1 = _f64(x1).reshape(-1)
    r = None if rho is None else _f64(rho).reshape(-1)
    toi = C.c_double(-1.0)
    hit = lib().orc_ccd(kind, _ptr(x0), _ptr(x1), _ptr(r) if r is not None else None, C.addressof(toi))
    return bool(hit), (toi.value if hit else None)


def ccd_conservative(kind, x0, x1, rho=None, tol=0.0):
    """True when the primitives may come within tol during the linear motion
    (False: certainly more than tol apart throughout)."""
    x0 = _f64(x0).reshape(-1)
    x1 = _f64(x1).reshape(-1)
    r = None if rho is None else _f64(rho).reshape(-1)
    return bool(lib().orc_ccd_conservative(kind, _ptr(x0), _ptr(x1), _ptr(r) if r is not None else None, tol))
