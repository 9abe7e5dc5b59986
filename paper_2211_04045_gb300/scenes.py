"""Seeded synthetic scenes and the stand-in dynamics that feeds each step.

This module produces inputs only: meshes, inverse masses, initial states and
the target ``x~`` of each step.  It holds none of the collision-handling
method's arithmetic, and serves both the CUDA path and the CPU oracle.

The paper's own meshes and animations are not available, so every scene is a
synthetic stand-in shaped like the paper's examples: cloth over a sphere, two
stacked cloth layers, a pile of volumetric bodies, two interleaved tubes that
tighten like a knot, and hair strands with sand grains in a bowl.

Frictional contact follows the paper's velocity filter (Sec. 6.3): a
pre-pass that turns each vertex-triangle contact's estimated penetration of
the frictionless target into a normal correction and a Coulomb-bounded
tangential one, before the collision-handling step.

A second workload is the globally injective normal flow of Sec. 7.4: the
target of each step is the surface pushed along its vertex normals and then
smoothed by three Jacobi steps of the cotangent Laplacian (Eq. normal flow);
the collision-handling step keeps the flow free of self-intersections.

The stand-in dynamics (not part of the method, which receives ``x~`` as
input) is explicit inertia ``x~ = x^t + dt v`` with scripted kinematic
vertices, followed by a few Jacobi sweeps that pull mesh edges toward their
rest lengths, and the velocity update ``v <- (x^{t+1} - x^t)/dt + dt g`` that
the paper uses to chain steps.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np


@dataclasses.dataclass
class Scene:
    name: str
    inv_mass: np.ndarray            # (n,) float64; 0 = fixed or kinematic
    tris: np.ndarray                # (T,3) int32 collision triangles
    edges: np.ndarray               # (E,2) int32 collision edges (edge-edge pairs)
    len_edges: np.ndarray           # (C,2) int32 edge-length constraints
    points: np.ndarray              # (Q,) int32 point participants (vertex-vertex pairs)
    x0: np.ndarray                  # (n,3) float64 initial, intersection-free
    v0: np.ndarray                  # (n,3) float64 initial velocity
    dt: float
    gravity: np.ndarray             # (3,)
    radius: Optional[np.ndarray] = None     # (n,) or None
    kin_v: Optional[np.ndarray] = None      # (n,3) scripted velocity of inv_mass==0 vertices
    rest_len: Optional[np.ndarray] = None   # (C,) rest lengths for the stand-in relaxation
    relax_sweeps: int = 4
    steps: int = 30
    params: dict = dataclasses.field(default_factory=dict)
    flow: Optional[dict] = None             # normal-flow target instead of the dynamics (beta, alpha, sign, iters)
    kin_rot: Optional[tuple] = None         # (angular velocity (3,), centre (3,)): kinematic vertices rotate
    friction: Optional[dict] = None         # velocity filter on the target (mu, reach, sep)

    @property
    def n_verts(self) -> int:
        return int(self.x0.shape[0])

    def counts(self) -> dict:
        return dict(verts=self.n_verts, tris=len(self.tris), edges=len(self.edges), len_edges=len(self.len_edges),
                    points=len(self.points))


# --------------------------------------------------------------------------
# mesh builders
# --------------------------------------------------------------------------
def unique_edges(tris: np.ndarray) -> np.ndarray:
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]], axis=0)
    e = np.sort(e, axis=1)
    e = np.unique(e, axis=0)
    return e.astype(np.int32)


def grid_cloth(n: int, side: float, height: float, center=(0.0, 0.0)):
    """n x n vertices spanning side x side in the xz plane at y = height."""
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    h = side / (n - 1)
    x = np.stack([center[0] - side / 2 + i * h, np.full(i.shape, height, dtype=np.float64),
                  center[1] - side / 2 + j * h], axis=-1).reshape(-1, 3)
    ii, jj = np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="ij")
    v00 = (ii * n + jj).ravel()
    v10 = ((ii + 1) * n + jj).ravel()
    v01 = (ii * n + jj + 1).ravel()
    v11 = ((ii + 1) * n + jj + 1).ravel()
    tris = np.concatenate([np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)], 0).astype(np.int32)
    return x.astype(np.float64), tris


def icosphere(subdiv: int, radius: float, center=(0.0, 0.0, 0.0)):
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6),
         (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10),
         (8, 6, 7), (9, 8, 1)]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = list(f)
    for _ in range(subdiv):
        cache = {}

        def mid(a, b):
            k = (min(a, b), max(a, b))
            if k not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[k] = len(verts) - 1
            return cache[k]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    x = np.array(verts) * radius + np.asarray(center, dtype=np.float64)
    return x, np.array(faces, dtype=np.int32)


def tet_cube(n: int, side: float):
    """n^3 vertex cube split into 6 Kuhn tetrahedra per cell (centred at 0)."""
    g = np.arange(n)
    i, j, k = np.meshgrid(g, g, g, indexing="ij")
    x = np.stack([i, j, k], -1).reshape(-1, 3).astype(np.float64) * (side / (n - 1)) - side / 2

    def vid(a, b, c):
        return (a * n + b) * n + c

    tets = []
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    for a in range(n - 1):
        for b in range(n - 1):
            for c in range(n - 1):
                base = np.array([a, b, c])
                for p in perms:
                    cur = base.copy()
                    tet = [vid(*cur)]
                    for ax in p:
                        cur = cur.copy()
                        cur[ax] += 1
                        tet.append(vid(*cur))
                    tets.append(tet)
    tets = np.array(tets, dtype=np.int64)
    faces = np.concatenate([tets[:, [0, 1, 2]], tets[:, [0, 1, 3]], tets[:, [0, 2, 3]], tets[:, [1, 2, 3]]], 0)
    fs = np.sort(faces, axis=1)
    uniq, inv, cnt = np.unique(fs, axis=0, return_inverse=True, return_counts=True)
    surface = uniq[cnt == 1].astype(np.int32)
    tet_edges = np.concatenate([tets[:, [a, b]] for a in range(4) for b in range(a + 1, 4)], 0)
    tet_edges = np.unique(np.sort(tet_edges, axis=1), axis=0).astype(np.int32)
    return x, tets.astype(np.int32), surface, tet_edges


def lumped_tri_mass(x, tris, n, density=1.0):
    a = x[tris[:, 1]] - x[tris[:, 0]]
    b = x[tris[:, 2]] - x[tris[:, 0]]
    area = 0.5 * np.linalg.norm(np.cross(a, b), axis=1)
    m = np.zeros(n)
    for k in range(3):
        m += np.bincount(tris[:, k], weights=area / 3.0 * density, minlength=n)
    return m


def lumped_tet_mass(x, tets, n, density=1.0):
    a = x[tets[:, 1]] - x[tets[:, 0]]
    b = x[tets[:, 2]] - x[tets[:, 0]]
    c = x[tets[:, 3]] - x[tets[:, 0]]
    vol = np.abs(np.einsum("ij,ij->i", a, np.cross(b, c))) / 6.0
    m = np.zeros(n)
    for k in range(4):
        m += np.bincount(tets[:, k], weights=vol / 4.0 * density, minlength=n)
    return m


def random_rotation(rng) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def _rest(x, len_edges):
    return np.linalg.norm(x[len_edges[:, 0]] - x[len_edges[:, 1]], axis=1)


# --------------------------------------------------------------------------
# scenes
# --------------------------------------------------------------------------
def cloth_over_sphere(n: int = 32, side: float = 1.0, sphere_subdiv: int = 3, sphere_r: float = 0.3,
                      gap: float = 0.05, seed: int = 0, noise: float = 0.5, v_down: float = 3.0,
                      dt: float = 1.0 / 30, steps: int = 30) -> Scene:
    """Cloth held horizontally `gap` above a fixed icosphere, thrown down onto it."""
    xc, tc = grid_cloth(n, side, sphere_r + gap)
    xs, ts = icosphere(sphere_subdiv, sphere_r)
    nc = len(xc)
    x = np.concatenate([xc, xs], 0)
    tris = np.concatenate([tc, ts + nc], 0).astype(np.int32)
    edges = unique_edges(tris)
    len_edges = unique_edges(tc)
    m = lumped_tri_mass(xc, tc, nc)
    inv_mass = np.concatenate([1.0 / m, np.zeros(len(xs))])
    rng = np.random.default_rng(seed)
    v = np.zeros_like(x)
    v[:nc] = np.array([0.0, -v_down, 0.0]) + rng.normal(0.0, noise, size=(nc, 3))
    return Scene(f"cloth{n}_sphere{sphere_subdiv}", inv_mass, tris, edges, len_edges, np.zeros(0, np.int32), x, v,
                 dt, np.array([0.0, -9.8, 0.0]), kin_v=np.zeros_like(x), rest_len=_rest(x, len_edges),
                 steps=steps, params=dict(max_iters=2048))


def two_cloths(n: int = 256, side: float = 2.0, sep: float = 0.01, omega: float = 6.0, noise: float = 0.3,
               seed: int = 0, dt: float = 1.0 / 30, steps: int = 60) -> Scene:
    """Two stacked n x n cloth grids `sep` apart; the top one spins about the vertical axis."""
    xb, tb = grid_cloth(n, side, 0.0)
    xt, tt = grid_cloth(n, side, sep)
    nb = len(xb)
    x = np.concatenate([xb, xt], 0)
    tris = np.concatenate([tb, tt + nb], 0).astype(np.int32)
    edges = unique_edges(tris)
    m = lumped_tri_mass(xb, tb, nb)
    inv_mass = np.concatenate([1.0 / m, 1.0 / m])
    rng = np.random.default_rng(seed)
    v = np.zeros_like(x)
    rel = xt - np.array([0.0, sep, 0.0])
    v[nb:, 0] = omega * rel[:, 2]
    v[nb:, 2] = -omega * rel[:, 0]
    v[nb:] += rng.normal(0.0, noise, size=(nb, 3))
    return Scene(f"two_cloths{n}", inv_mass, tris, edges, edges.copy(), np.zeros(0, np.int32), x, v, dt,
                 np.zeros(3), kin_v=np.zeros_like(x), rest_len=_rest(x, edges), steps=steps,
                 params=dict(max_iters=2048))


def tet_bodies(n_bodies: int = 64, n: int = 8, side: float = 0.2, box: float = 1.5, seed: int = 0,
               v_sigma: float = 2.0, w_sigma: float = 4.0, dt: float = 1.0 / 20, steps: int = 100) -> Scene:
    """Cube tet meshes at random orientations on a lattice inside a `box` cube."""
    xb, tets, surf, tedges = tet_cube(n, side)
    k = int(math.ceil(n_bodies ** (1.0 / 3.0) - 1e-9))
    spacing = box / k
    if spacing < side * math.sqrt(3.0):
        raise ValueError("bodies would overlap")
    rng = np.random.default_rng(seed)
    nb = len(xb)
    xs, vs, tr, ed, le, tt = [], [], [], [], [], []
    surf_edges = unique_edges(surf)
    mb = lumped_tet_mass(xb, tets, nb)
    for b in range(n_bodies):
        c = np.array([(b % k + 0.5), ((b // k) % k + 0.5), (b // (k * k) + 0.5)]) * spacing
        R = random_rotation(rng)
        xw = xb @ R.T + c
        vl = rng.normal(0.0, v_sigma, size=3)
        w = rng.normal(0.0, w_sigma, size=3)
        xs.append(xw)
        vs.append(vl + np.cross(w, xw - c))
        tr.append(surf + b * nb)
        ed.append(surf_edges + b * nb)
        le.append(tedges + b * nb)
        tt.append(tets + b * nb)
    x = np.concatenate(xs, 0)
    v = np.concatenate(vs, 0)
    inv_mass = np.tile(1.0 / mb, n_bodies)
    len_edges = np.concatenate(le, 0).astype(np.int32)
    return Scene(f"tets{n_bodies}x{n}", inv_mass, np.concatenate(tr, 0).astype(np.int32),
                 np.concatenate(ed, 0).astype(np.int32), len_edges, np.zeros(0, np.int32), x, v, dt, np.zeros(3),
                 kin_v=np.zeros_like(x), rest_len=_rest(x, len_edges), steps=steps, params=dict(max_iters=2048))


def tube_knot(around: int = 64, rings: int = 561, r: float = 0.01, helix_r: float = 0.012, pitch: float = 0.04,
              ring_dz: float = 0.0015, pull: float = 1.0, dt: float = 1.0 / 30, steps: int = 200) -> Scene:
    """Two open tubes wound around each other as a double helix; the end rings
    are kinematic and pulled apart along the axis so the twist tightens."""
    xs, ts = [], []
    kin = []
    length = (rings - 1) * ring_dz
    for s in range(2):
        phase = math.pi * s
        zc = np.arange(rings) * ring_dz - length / 2
        ang = 2 * math.pi * (zc + length / 2) / pitch + phase
        cx, cy = helix_r * np.cos(ang), helix_r * np.sin(ang)
        th = 2 * math.pi * np.arange(around) / around
        px = cx[:, None] + r * np.cos(th)[None, :]
        py = cy[:, None] + r * np.sin(th)[None, :]
        pz = np.broadcast_to(zc[:, None], px.shape)
        x = np.stack([px, py, pz], -1).reshape(-1, 3)
        a = np.arange(rings - 1)[:, None]
        b = np.arange(around)[None, :]
        v00 = a * around + b
        v01 = a * around + (b + 1) % around
        v10 = (a + 1) * around + b
        v11 = (a + 1) * around + (b + 1) % around
        t = np.concatenate([np.stack([v00, v10, v11], -1).reshape(-1, 3), np.stack([v00, v11, v01], -1).reshape(-1, 3)])
        base = s * rings * around
        xs.append(x)
        ts.append(t + base)
        kin.append(np.arange(around) + base)
        kin.append(np.arange((rings - 1) * around, rings * around) + base)
    x = np.concatenate(xs, 0)
    tris = np.concatenate(ts, 0).astype(np.int32)
    edges = unique_edges(tris)
    n = len(x)
    m = lumped_tri_mass(x, tris, n)
    inv_mass = 1.0 / m
    kin_v = np.zeros_like(x)
    for s in range(2):
        lo = s * rings * around
        kin_v[lo:lo + around, 2] = -pull
        kin_v[lo + (rings - 1) * around: lo + rings * around, 2] = pull
        inv_mass[lo:lo + around] = 0.0
        inv_mass[lo + (rings - 1) * around: lo + rings * around] = 0.0
    v = kin_v.copy()
    return Scene(f"knot{around}x{rings}", inv_mass, tris, edges, edges.copy(), np.zeros(0, np.int32), x, v, dt,
                 np.zeros(3), kin_v=kin_v, rest_len=_rest(x, edges), relax_sweeps=10, steps=steps,
                 params=dict(max_iters=2048, delta=0.5e-3, d_min=1e-3, d_max=2e-3))


def hair_sand(n_strands: int = 10000, segs: int = 32, n_points: int = 100000, grain_r: float = 0.002,
              bowl_r: float = 0.5, bowl_subdiv: int = 5, seg_len: float = 0.01, seed: int = 0,
              dt: float = 1.0 / 30, steps: int = 200) -> Scene:
    """Hair strands and sand grains poured from a lattice above a fixed bowl."""
    rng = np.random.default_rng(seed)
    xs_b, ts_b = icosphere(bowl_subdiv, bowl_r)
    keep = xs_b[:, 1] < 1e-9
    fk = np.all(keep[ts_b], axis=1)
    ts_b = ts_b[fk]
    used = np.unique(ts_b)
    remap = -np.ones(len(xs_b), np.int64)
    remap[used] = np.arange(len(used))
    xb = xs_b[used] + np.array([0.0, bowl_r, 0.0])
    tb = remap[ts_b].astype(np.int32)
    # strands hang vertically on a square lattice above the bowl
    sq = int(math.ceil(math.sqrt(n_strands)))
    span = 0.6 * bowl_r
    gx = (np.arange(sq) + 0.5) / sq * 2 * span - span
    sx, sz = np.meshgrid(gx, gx, indexing="ij")
    roots = np.stack([sx.ravel(), sz.ravel()], -1)[:n_strands]
    top = bowl_r + 0.05 + segs * seg_len
    hx = []
    for k in range(segs + 1):
        hx.append(np.stack([roots[:, 0], np.full(len(roots), top - k * seg_len), roots[:, 1]], -1))
    hx = np.stack(hx, 1).reshape(-1, 3)
    nh = len(hx)
    sid = np.arange(n_strands)[:, None] * (segs + 1)
    se = np.stack([sid + np.arange(segs)[None, :], sid + np.arange(1, segs + 1)[None, :]], -1).reshape(-1, 2)
    # sand grains on a lattice above the strands
    pc = int(math.ceil(n_points ** (1.0 / 3.0)))
    pitch = 3.0 * grain_r
    g = (np.arange(pc) - (pc - 1) / 2) * pitch
    px, py, pz = np.meshgrid(g, np.arange(pc) * pitch, g, indexing="ij")
    pts = np.stack([px.ravel(), py.ravel() + top + 0.02, pz.ravel()], -1)[:n_points]
    nb = len(xb)
    x = np.concatenate([xb, hx, pts], 0)
    n = len(x)
    tris = tb
    edges = np.concatenate([unique_edges(tb), se + nb], 0).astype(np.int32)
    points = (np.arange(len(pts)) + nb + nh).astype(np.int32)
    inv_mass = np.concatenate([np.zeros(nb), np.full(nh, 1.0 / (seg_len * 1.0)), np.full(len(pts), 1.0)])
    radius = np.concatenate([np.zeros(nb + nh), np.full(len(pts), grain_r)])
    v = np.zeros_like(x)
    v[nb:] = np.array([0.0, -2.0, 0.0]) + rng.normal(0.0, 0.2, size=(n - nb, 3))
    len_edges = (se + nb).astype(np.int32)
    return Scene(f"hair{n_strands}x{segs}_sand{n_points}", inv_mass, tris, edges, len_edges, points, x, v, dt,
                 np.array([0.0, -9.8, 0.0]), radius=radius, kin_v=np.zeros_like(x), rest_len=_rest(x, len_edges),
                 steps=steps, params=dict(max_iters=2048, delta=0.2e-3, d_min=0.4e-3, d_max=0.8e-3))


# --------------------------------------------------------------------------
# stand-in dynamics that produces x~ for each step
# --------------------------------------------------------------------------
# --------------------------------------------------------------------------
# globally injective normal flow (Sec. 7.4, Eq. normal flow)
# --------------------------------------------------------------------------
def torus_mesh(n_major: int, n_minor: int, R: float, r: float):
    """Closed torus around the z axis: n_major rings of n_minor vertices;
    triangles wound so that (b - a) x (c - a) points outward."""
    u = 2 * math.pi * np.arange(n_major) / n_major
    w = 2 * math.pi * np.arange(n_minor) / n_minor
    U, W = np.meshgrid(u, w, indexing="ij")
    A = R + r * np.cos(W)
    x = np.stack([A * np.cos(U), A * np.sin(U), r * np.sin(W)], -1).reshape(-1, 3)
    i, j = np.meshgrid(np.arange(n_major), np.arange(n_minor), indexing="ij")
    v00 = i * n_minor + j
    v10 = ((i + 1) % n_major) * n_minor + j
    v11 = ((i + 1) % n_major) * n_minor + (j + 1) % n_minor
    v01 = i * n_minor + (j + 1) % n_minor
    tris = np.concatenate([np.stack([v00, v10, v11], -1).reshape(-1, 3),
                           np.stack([v00, v11, v01], -1).reshape(-1, 3)]).astype(np.int32)
    return x, tris


def vertex_normals(x: np.ndarray, tris: np.ndarray) -> np.ndarray:
    """Unit vertex normals: the area-weighted sum of the incident faces'
    normals (each face adds (b - a) x (c - a), twice its area times its unit
    normal)."""
    a, b, c = x[tris[:, 0]], x[tris[:, 1]], x[tris[:, 2]]
    fn = np.cross(b - a, c - a)
    n = np.zeros_like(x)
    for k in range(3):
        np.add.at(n, tris[:, k], fn)
    L = np.linalg.norm(n, axis=1)
    return n / np.where(L > 0, L, 1.0)[:, None]


def cotan_laplacian(y: np.ndarray, tris: np.ndarray) -> np.ndarray:
    """Cotangent discretisation of the Laplace-Beltrami operator applied to
    the coordinates y: (Lap y)(v) = 1/(2 A_v) sum_u (cot a_vu + cot b_vu)
    (y_u - y_v), with A_v the mixed Voronoi area of Meyer et al. (2003): a
    corner of a non-obtuse triangle takes its Voronoi part, (|e1|^2 cot +
    |e2|^2 cot)/8 over its two edges and their opposite angles; in an obtuse
    triangle the obtuse corner takes half the area and the others a quarter."""
    p = [y[tris[:, k]] for k in range(3)]
    n = np.zeros_like(y)
    A = np.zeros(len(y))
    area2 = np.linalg.norm(np.cross(p[1] - p[0], p[2] - p[0]), axis=1)
    safe2 = np.where(area2 > 0, area2, 1.0)
    dots = [np.einsum("ij,ij->i", p[(k + 1) % 3] - p[k], p[(k + 2) % 3] - p[k]) for k in range(3)]
    cot = [d / safe2 for d in dots]
    obtuse = (dots[0] < 0) | (dots[1] < 0) | (dots[2] < 0)
    for k in range(3):
        q, s_ = p[(k + 1) % 3], p[(k + 2) % 3]
        # the edge (q, s) opposite corner k carries cot/2 to both its ends
        np.add.at(n, tris[:, (k + 1) % 3], 0.5 * cot[k][:, None] * (s_ - q))
        np.add.at(n, tris[:, (k + 2) % 3], 0.5 * cot[k][:, None] * (q - s_))
        e_q = np.einsum("ij,ij->i", q - p[k], q - p[k])    # edge k-(k+1), opposite corner k+2
        e_s = np.einsum("ij,ij->i", s_ - p[k], s_ - p[k])  # edge k-(k+2), opposite corner k+1
        vor = (e_q * cot[(k + 2) % 3] + e_s * cot[(k + 1) % 3]) / 8.0
        np.add.at(A, tris[:, k], np.where(~obtuse, vor, np.where(dots[k] < 0, area2 / 4.0, area2 / 8.0)))
    return n / np.where(A > 0, A, 1.0)[:, None]


def normal_flow_target(x: np.ndarray, tris: np.ndarray, beta: float, alpha: float, sign: float = 1.0,
                       iters: int = 3) -> np.ndarray:
    """Eq. normal flow: y_0 = x + sign beta n(x), then `iters` Jacobi steps
    y_{i+1} = y_i + alpha Lap(y_i), the operator taken on the surface y_i."""
    y = x + (sign * beta) * vertex_normals(x, tris)
    for _ in range(iters):
        y = y + alpha * cotan_laplacian(y, tris)
    return y


def normal_flow_torus(n_major: int = 384, n_minor: int = 64, R: float = 0.1, r: float = 0.012,
                      beta: float = 2e-3, alpha_frac: float = 0.1, sign: float = -1.0, steps: int = 8) -> Scene:
    """A closed torus under the normal flow of Sec. 7.4 (the paper's meshes
    are not available).  sign = -1 shrinks the tube until its opposite sides
    meet; sign = +1 with R - r small closes the hole.  alpha is alpha_frac
    times the squared mean edge length (the explicit Jacobi step is stable
    well below 1/4 of it)."""
    x, tris = torus_mesh(n_major, n_minor, R, r)
    edges = unique_edges(tris)
    h = float(np.mean(np.linalg.norm(x[edges[:, 0]] - x[edges[:, 1]], axis=1)))
    flow = dict(beta=beta, alpha=alpha_frac * h * h, sign=sign, iters=3)
    n = len(x)
    return Scene(f"normal_flow_torus{n_major}x{n_minor}{'+' if sign > 0 else '-'}", np.ones(n), tris, edges,
                 edges.copy(), np.zeros(0, np.int32), x, np.zeros_like(x), 1.0, np.zeros(3), relax_sweeps=0,
                 steps=steps, params=dict(max_iters=2048), flow=flow)


# --------------------------------------------------------------------------
# friction by velocity filtering (Sec. 6.3, after Bridson et al. 2002)
# --------------------------------------------------------------------------
def rotate(p: np.ndarray, rotvec: np.ndarray, centre) -> np.ndarray:
    """Rodrigues rotation of the rows of p by the rotation vector rotvec
    about an axis through centre."""
    c = np.asarray(centre, dtype=np.float64)
    th = float(np.linalg.norm(rotvec))
    if th == 0.0:
        return p.copy()
    k = np.asarray(rotvec, dtype=np.float64) / th
    q = p - c
    kq = np.cross(k, q)
    return c + q * math.cos(th) + kq * math.sin(th) + np.outer(q @ k, k) * (1.0 - math.cos(th))


def closest_on_triangle(p, a, b, c):
    """Closest points of the triangles (a, b, c) to the points p (one per
    row) as barycentric weights, by the Voronoi regions of the triangle:
    the three corners, the three edges, else the interior (Ericson,
    Real-Time Collision Detection, Sec. 5.1.5)."""
    ab, ac = b - a, c - a
    dot = lambda u, w: np.einsum("ij,ij->i", u, w)  # noqa: E731
    ap, bp, cp = p - a, p - b, p - c
    d1, d2 = dot(ab, ap), dot(ac, ap)
    d3, d4 = dot(ab, bp), dot(ac, bp)
    d5, d6 = dot(ab, cp), dot(ac, cp)
    va, vb, vc = d3 * d6 - d5 * d4, d5 * d2 - d1 * d6, d1 * d4 - d3 * d2
    n = len(p)
    w = np.zeros((n, 3))
    done = np.zeros(n, bool)

    def put(mask, w0, w1, w2):
        m = mask & ~done
        w[m, 0], w[m, 1], w[m, 2] = w0[m], w1[m], w2[m]
        done[m] = True

    one, zero = np.ones(n), np.zeros(n)
    put((d1 <= 0) & (d2 <= 0), one, zero, zero)
    put((d3 >= 0) & (d4 <= d3), zero, one, zero)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = d1 / (d1 - d3)
        put((vc <= 0) & (d1 >= 0) & (d3 <= 0), 1 - t, t, zero)
        put((d6 >= 0) & (d5 <= d6), zero, zero, one)
        t = d2 / (d2 - d6)
        put((vb <= 0) & (d2 >= 0) & (d6 <= 0), 1 - t, zero, t)
        t = (d4 - d3) / ((d4 - d3) + (d5 - d6))
        put((va <= 0) & (d4 - d3 >= 0) & (d5 - d6 >= 0), zero, 1 - t, t)
        den = va + vb + vc
        v_, w_ = vb / den, vc / den
        put(np.ones(n, bool), 1 - v_ - w_, v_, w_)
    return w


def friction_filter(x: np.ndarray, y: np.ndarray, inv_mass: np.ndarray, tris: np.ndarray, mu: float,
                    reach: float, sep: float) -> np.ndarray:
    """Velocity filter of Sec. 6.3 on the frictionless target y.

    Every vertex-triangle pair closer than `reach` at x (any vertex; the triangle not
    containing the vertex, not all four vertices fixed) is a contact with
    normal n from the triangle's closest point to the vertex.  Its relative
    displacement u = (y_p - x_p) - sum_i w_i (y_i - x_i) would leave it at
    separation d + n.u; the penetration depth pen = sep - (d + n.u) > 0 is
    the collision impulse (as a displacement along n), and Coulomb's law
    bounds the friction impulse, which opposes the tangential part u_t, by
    mu pen.  The pair's relative correction pen n - min(mu pen, |u_t|)
    u_t/|u_t| is shared by inverse mass (vertex m_p^-1 / W, triangle vertex i
    -w_i m_i^-1 / W, W = m_p^-1 + sum w_i^2 m_i^-1), which keeps the momentum
    sum m Delta at zero.  A vertex in several contacts takes the mean of its
    corrections (a Jacobi pass, independent of the pair order)."""
    from scipy.spatial import cKDTree
    tris = np.asarray(tris, np.int64)
    n = len(x)
    if len(tris) == 0:
        return y.copy()
    a, b, c = x[tris[:, 0]], x[tris[:, 1]], x[tris[:, 2]]
    cen = (a + b + c) / 3.0
    rad = np.max(np.stack([np.linalg.norm(q - cen, axis=1) for q in (a, b, c)], 1), axis=1)
    verts = np.arange(n)
    lists = cKDTree(cen).query_ball_point(x[verts], reach + float(rad.max()))
    pv = np.repeat(verts, [len(l) for l in lists])
    pt = np.fromiter((t for l in lists for t in l), np.int64, count=len(pv))
    if len(pv) == 0:
        return y.copy()
    tv = tris[pt]
    keep = (tv != pv[:, None]).all(1)
    keep &= (inv_mass[pv] > 0) | (inv_mass[tv] > 0).any(1)
    pv, tv = pv[keep], tv[keep]
    P, A, B, C = x[pv], x[tv[:, 0]], x[tv[:, 1]], x[tv[:, 2]]
    w = closest_on_triangle(P, A, B, C)
    q = w[:, :1] * A + w[:, 1:2] * B + w[:, 2:] * C
    d = np.linalg.norm(P - q, axis=1)
    near = (d < reach) & (d > 0)
    pv, tv, w, d, P, q = pv[near], tv[near], w[near], d[near], P[near], q[near]
    nrm = (P - q) / d[:, None]
    dy = y - x
    u = dy[pv] - np.einsum("ij,ijk->ik", w, dy[tv])
    un = np.einsum("ij,ij->i", u, nrm)
    pen = sep - (d + un)
    W = inv_mass[pv] + np.einsum("ij,ij->i", w * w, inv_mass[tv])
    act = (pen > 0) & (W > 0)
    pv, tv, w, nrm, u, un, pen, W = pv[act], tv[act], w[act], nrm[act], u[act], un[act], pen[act], W[act]
    ut = u - un[:, None] * nrm
    lt = np.linalg.norm(ut, axis=1)
    f = np.minimum(mu * pen, lt)
    du = pen[:, None] * nrm - (f / np.where(lt > 0, lt, 1.0))[:, None] * ut
    corr = np.zeros_like(y)
    cnt = np.zeros(n)
    np.add.at(corr, pv, (inv_mass[pv] / W)[:, None] * du)
    np.add.at(cnt, pv, inv_mass[pv] > 0)
    for k in range(3):
        vi = tv[:, k]
        np.add.at(corr, vi, -(w[:, k] * inv_mass[vi] / W)[:, None] * du)
        np.add.at(cnt, vi, (inv_mass[vi] > 0) & (w[:, k] != 0))
    return y + corr / np.maximum(cnt, 1.0)[:, None]


def cloth_on_rotating_sphere(n: int = 32, side: float = 1.0, sphere_subdiv: int = 3, sphere_r: float = 0.3,
                             gap: float = 0.002, omega: float = 2.0, mu: float = 0.5, dt: float = 1.0 / 30,
                             steps: int = 30) -> Scene:
    """The rotating-sphere example of Sec. 6.3: a cloth resting on a sphere
    that spins about the vertical axis; the velocity filter makes the sphere
    drag the cloth (without it the cloth slides)."""
    xc, tc = grid_cloth(n, side, sphere_r + gap)
    xs, ts = icosphere(sphere_subdiv, sphere_r)
    nc = len(xc)
    x = np.concatenate([xc, xs], 0)
    tris = np.concatenate([tc, ts + nc], 0).astype(np.int32)
    edges = unique_edges(tris)
    len_edges = unique_edges(tc)
    m = lumped_tri_mass(xc, tc, nc)
    inv_mass = np.concatenate([1.0 / m, np.zeros(len(xs))])
    return Scene(f"cloth{n}_rotating_sphere{sphere_subdiv}", inv_mass, tris, edges, len_edges,
                 np.zeros(0, np.int32), x, np.zeros_like(x), dt, np.array([0.0, -9.8, 0.0]),
                 rest_len=_rest(x, len_edges), steps=steps, params=dict(max_iters=2048),
                 kin_rot=(np.array([0.0, omega, 0.0]), np.zeros(3)),
                 friction=dict(mu=mu, reach=2e-3, sep=1e-3) if mu > 0 else None)


def predict(scene: Scene, x: np.ndarray, v: np.ndarray) -> np.ndarray:
    """x~ = x + dt v, kinematic vertices on their script, then Jacobi
    sweeps toward rest edge lengths (inverse-mass weighted).  A normal-flow
    scene ignores v: its target is Eq. normal flow at x."""
    if scene.flow is not None:
        return normal_flow_target(x, scene.tris, **scene.flow)
    xt = x + scene.dt * v
    im = scene.inv_mass
    fixed = im == 0.0
    if scene.kin_v is not None:
        xt[fixed] = x[fixed] + scene.dt * scene.kin_v[fixed]
    if scene.kin_rot is not None:
        w, c = scene.kin_rot
        xt[fixed] = rotate(x[fixed], np.asarray(w) * scene.dt, c)
    le = scene.len_edges
    if scene.relax_sweeps and len(le) and scene.rest_len is not None:
        n = len(x)
        i, j = le[:, 0], le[:, 1]
        wi, wj = im[i], im[j]
        ws = wi + wj
        ok = ws > 0
        deg = np.bincount(i[ok], minlength=n) + np.bincount(j[ok], minlength=n)
        deg = np.maximum(deg, 1).astype(np.float64)
        for _ in range(scene.relax_sweeps):
            d = xt[i] - xt[j]
            L = np.linalg.norm(d, axis=1)
            L = np.where(L > 0, L, 1.0)
            corr = np.where(ok, (L - scene.rest_len) / L / np.where(ok, ws, 1.0), 0.0)[:, None] * d
            dx = np.zeros_like(xt)
            for k in range(3):
                dx[:, k] -= np.bincount(i, weights=wi * corr[:, k], minlength=n)
                dx[:, k] += np.bincount(j, weights=wj * corr[:, k], minlength=n)
            xt += dx / deg[:, None]
    if scene.friction is not None:
        xt = friction_filter(x, xt, im, scene.tris, **scene.friction)
    return xt


def next_velocity(scene: Scene, x_new: np.ndarray, x_old: np.ndarray) -> np.ndarray:
    v = (x_new - x_old) / scene.dt
    movable = scene.inv_mass > 0
    v[movable] += scene.dt * scene.gravity
    if scene.kin_v is not None:
        v[~movable] = scene.kin_v[~movable]
    return v


def initial(scene: Scene):
    """(x^0, x~^0) of the first step."""
    x = scene.x0.copy()
    v = scene.v0.copy()
    v[scene.inv_mass > 0] += scene.dt * scene.gravity
    return x, predict(scene, x, v), v


def by_name(name: str, **kw) -> Scene:
    table = {
        "cloth_sphere": cloth_over_sphere,
        "two_cloths": two_cloths,
        "tets": tet_bodies,
        "knot": tube_knot,
        "hair_sand": hair_sand,
        "normal_flow": normal_flow_torus,
        "rotating_sphere": cloth_on_rotating_sphere,
    }
    return table[name](**kw)


# --------------------------------------------------------------------------
# the same stand-in dynamics on the GPU (torch), used by the benchmark to
# chain steps without host round trips
# --------------------------------------------------------------------------
class TorchDynamics:
    def __init__(self, scene: Scene, device):
        import torch
        self.torch = torch
        self.sc = scene
        f = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=device)  # noqa: E731
        if scene.flow is not None:
            # per-vertex table of (triangle, corner) slots, padded with a
            # zero slot: the per-vertex sums of the normal flow run in a
            # fixed order, without atomics
            t = scene.tris.astype(np.int64)
            n, T = scene.n_verts, len(t)
            ends = t.reshape(-1)
            slots = np.arange(3 * T)
            order = np.argsort(ends, kind="stable")
            ends, slots = ends[order], slots[order]
            cnt = np.bincount(ends, minlength=n)
            width = max(1, int(cnt.max()))
            start = np.concatenate([[0], np.cumsum(cnt)[:-1]])
            col = np.arange(len(ends)) - start[ends]
            idx = np.full((n, width), 3 * T, np.int64)
            idx[ends, col] = slots
            self.f_tris = f(t)
            self.f_slot = f(idx)
        self.im = f(scene.inv_mass)
        self.fixed = self.im == 0.0
        self.kin_v = f(scene.kin_v if scene.kin_v is not None else np.zeros_like(scene.x0))
        self.g = f(scene.gravity)
        le = scene.len_edges
        self.relax = bool(scene.relax_sweeps and len(le) and scene.rest_len is not None)
        if self.relax:
            self.i = f(le[:, 0].astype(np.int64))
            self.j = f(le[:, 1].astype(np.int64))
            wi, wj = self.im[self.i], self.im[self.j]
            ws = wi + wj
            self.ok = ws > 0
            self.wi, self.wj = wi, wj
            self.ws = torch.where(self.ok, ws, torch.ones_like(ws))
            n, m = scene.n_verts, len(le)
            im = scene.inv_mass
            ok = (im[le[:, 0]] + im[le[:, 1]]) > 0
            deg = np.maximum(np.bincount(le[ok, 0], minlength=n) + np.bincount(le[ok, 1], minlength=n), 1)
            self.deg = f(deg.astype(np.float64))[:, None]
            # per-vertex incidence table (edge row, weight), padded with a
            # zero row: the per-vertex sums then run in a fixed order and the
            # prediction is bitwise reproducible (no atomic accumulation)
            ends = np.concatenate([le[:, 0], le[:, 1]])
            rows = np.concatenate([np.arange(m), np.arange(m)])
            wts = np.concatenate([-im[le[:, 0]], im[le[:, 1]]])
            order = np.argsort(ends, kind="stable")
            ends, rows, wts = ends[order], rows[order], wts[order]
            cnt = np.bincount(ends, minlength=n)
            width = max(1, int(cnt.max()) if len(cnt) else 1)
            start = np.concatenate([[0], np.cumsum(cnt)[:-1]])
            slot = np.arange(len(ends)) - start[ends]
            idx = np.full((n, width), m, np.int64)
            w = np.zeros((n, width))
            idx[ends, slot] = rows
            w[ends, slot] = wts
            self.inc_idx, self.inc_w = f(idx), f(w)[:, :, None]
            self.rest = f(scene.rest_len)

    def _gather(self, per_corner):
        # per_corner: (T, 3, ...) values of each triangle corner -> per-vertex sums
        flat = per_corner.reshape(-1, *per_corner.shape[2:])
        flat = self.torch.cat([flat, self.torch.zeros_like(flat[:1])])
        return flat[self.f_slot].sum(dim=1)

    def _flow(self, x):
        torch = self.torch
        fl = self.sc.flow
        t = self.f_tris
        p = [x[t[:, k]] for k in range(3)]
        fn = torch.linalg.cross(p[1] - p[0], p[2] - p[0])
        nv = self._gather(torch.stack([fn, fn, fn], 1))
        L = torch.linalg.norm(nv, dim=1, keepdim=True)
        y = x + (fl["sign"] * fl["beta"]) * (nv / torch.where(L > 0, L, torch.ones_like(L)))
        for _ in range(fl["iters"]):
            p = [y[t[:, k]] for k in range(3)]
            area2 = torch.linalg.norm(torch.linalg.cross(p[1] - p[0], p[2] - p[0]), dim=1)
            safe2 = torch.where(area2 > 0, area2, torch.ones_like(area2))
            dots = [((p[(k + 1) % 3] - p[k]) * (p[(k + 2) % 3] - p[k])).sum(1) for k in range(3)]
            cot = [d / safe2 for d in dots]
            obtuse = (dots[0] < 0) | (dots[1] < 0) | (dots[2] < 0)
            lap = [torch.zeros_like(p[0]) for _ in range(3)]
            area = []
            for k in range(3):
                q, s_ = p[(k + 1) % 3], p[(k + 2) % 3]
                lap[(k + 1) % 3] = lap[(k + 1) % 3] + 0.5 * cot[k][:, None] * (s_ - q)
                lap[(k + 2) % 3] = lap[(k + 2) % 3] + 0.5 * cot[k][:, None] * (q - s_)
                e_q = ((q - p[k]) ** 2).sum(1)
                e_s = ((s_ - p[k]) ** 2).sum(1)
                vor = (e_q * cot[(k + 2) % 3] + e_s * cot[(k + 1) % 3]) / 8.0
                area.append(torch.where(~obtuse, vor, torch.where(dots[k] < 0, area2 / 4.0, area2 / 8.0)))
            Lv = self._gather(torch.stack(lap, 1))
            Av = self._gather(torch.stack(area, 1))
            y = y + fl["alpha"] * (Lv / torch.where(Av > 0, Av, torch.ones_like(Av))[:, None])
        return y

    def _rotate(self, p, rotvec, centre):
        # Rodrigues rotation of the rows of p about an axis through centre
        torch = self.torch
        c = torch.as_tensor(np.asarray(centre, dtype=np.float64), device=p.device)
        th = float(np.linalg.norm(rotvec))
        if th == 0.0:
            return p.clone()
        k = torch.as_tensor(np.asarray(rotvec, dtype=np.float64) / th, device=p.device)
        q = p - c
        kq = torch.linalg.cross(k.expand_as(q), q)
        return c + q * math.cos(th) + kq * math.sin(th) + torch.outer(q @ k, k) * (1.0 - math.cos(th))

    def predict(self, x, v):
        if self.sc.friction is not None:
            raise NotImplementedError("the friction filter is a pre-pass of its own: use predict_frictionless "
                                      "and apply the filter to its result")
        return self.predict_frictionless(x, v)

    def predict_frictionless(self, x, v):
        torch = self.torch
        sc = self.sc
        if sc.flow is not None:
            return self._flow(x)
        xt = x + sc.dt * v
        xt = torch.where(self.fixed[:, None], x + sc.dt * self.kin_v, xt)
        if sc.kin_rot is not None:
            w, c = sc.kin_rot
            xt = torch.where(self.fixed[:, None], self._rotate(x, np.asarray(w) * sc.dt, c), xt)
        if self.relax:
            for _ in range(sc.relax_sweeps):
                d = xt[self.i] - xt[self.j]
                L = torch.linalg.norm(d, dim=1)
                L = torch.where(L > 0, L, torch.ones_like(L))
                c = torch.where(self.ok, (L - self.rest) / L / self.ws, torch.zeros_like(L))[:, None] * d
                c = torch.cat([c, torch.zeros_like(c[:1])])
                dx = (self.inc_w * c[self.inc_idx]).sum(dim=1)
                xt = xt + dx / self.deg
        return xt

    def next_velocity(self, x_new, x_old):
        torch = self.torch
        v = (x_new - x_old) / self.sc.dt
        v = torch.where(self.fixed[:, None], self.kin_v, v + self.sc.dt * self.g)
        return v
