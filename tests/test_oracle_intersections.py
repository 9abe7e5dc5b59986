"""Pins of the oracle's exact intersection count (the acceptance test of
x^{t+1} and the final check of P5): an independent brute force in exact
rational arithmetic on random generic configurations, and closed-form
touching cases (closed primitives count when they touch)."""
from fractions import Fraction
from types import SimpleNamespace as NS

import numpy as np
import pytest

import oracle


def orient(a, b, c, d):
    a, b, c, d = ([Fraction(float(v)) for v in p] for p in (a, b, c, d))
    u = [b[i] - a[i] for i in range(3)]
    v = [c[i] - a[i] for i in range(3)]
    w = [d[i] - a[i] for i in range(3)]
    det = (u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0]) +
           u[2] * (v[0] * w[1] - v[1] * w[0]))
    return (det > 0) - (det < 0)


def seg_tri_generic(p, q, a, b, c):
    s1, s2 = orient(a, b, c, p), orient(a, b, c, q)
    assert s1 != 0 and s2 != 0
    if s1 == s2:
        return 0
    t = [orient(p, q, a, b), orient(p, q, b, c), orient(p, q, c, a)]
    assert 0 not in t
    return int(all(v > 0 for v in t) or all(v < 0 for v in t))


def mesh(x, tris=(), edges=(), points=(), radius=None):
    return NS(n_verts=len(x), inv_mass=np.ones(len(x)), radius=radius, tris=np.asarray(tris, np.int32).reshape(-1, 3),
              edges=np.asarray(edges, np.int32).reshape(-1, 2), len_edges=np.zeros((0, 2), np.int32),
              points=np.asarray(points, np.int32))


@pytest.mark.parametrize("seed", range(10))
def test_random_segments_through_triangles(seed):
    rng = np.random.default_rng(seed)
    nt, ne = 6, 10
    x = rng.normal(0.0, 1.0, size=(3 * nt + 2 * ne, 3))
    tris = np.arange(3 * nt).reshape(nt, 3)
    edges = 3 * nt + np.arange(2 * ne).reshape(ne, 2)
    want = sum(seg_tri_generic(x[e[0]], x[e[1]], *x[t]) for e in edges for t in tris)
    got = oracle.count_intersections(oracle.OracleScene(mesh(x, tris, edges)), x)
    assert got == want and (seed > 0 or want > 0)


def test_touching_cases_count():
    tri = [[0.0, 0, 0], [1.0, 0, 0], [0, 1.0, 0]]
    cases = [
        ([[0.25, 0.25, 1.0], [0.25, 0.25, -1.0]], 1),    # through the interior
        ([[0.25, 0.25, 1.0], [0.25, 0.25, 0.0]], 1),     # endpoint on the triangle
        ([[0.5, 0.0, 1.0], [0.5, 0.0, -1.0]], 1),        # through an edge
        ([[0.0, 0.0, 1.0], [0.0, 0.0, -1.0]], 1),        # through a vertex (not shared)
        ([[-1.0, 0.5, 0.0], [2.0, 0.5, 0.0]], 1),        # coplanar, crossing
        ([[0.25, 0.25, 1.0], [0.25, 0.25, 1e-9]], 0),    # stops just short
        ([[0.8, 0.8, 1.0], [0.8, 0.8, -1.0]], 0),        # beside the hypotenuse
        ([[-1.0, 0.5, 1e-12], [2.0, 0.5, 1e-12]], 0),    # parallel, just above
    ]
    for seg, want in cases:
        x = np.array(tri + seg)
        sc = mesh(x, tris=[[0, 1, 2]], edges=[[3, 4]])
        assert oracle.count_intersections(oracle.OracleScene(sc), x) == want, seg


def test_edges_and_points():
    # crossing coplanar edges count, skew ones do not, touching collinear ones do
    x = np.array([[-1.0, 0, 0], [1.0, 0, 0], [0, -1.0, 0], [0, 1.0, 0], [0, -1.0, 1e-9], [0, 1.0, 1e-9],
                  [1.0, 0, 0.0], [3.0, 0, 0.0]])
    assert oracle.count_intersections(oracle.OracleScene(mesh(x, edges=[[0, 1], [2, 3]])), x) == 1
    assert oracle.count_intersections(oracle.OracleScene(mesh(x, edges=[[0, 1], [4, 5]])), x) == 0
    xs = x.copy()
    xs[6] = [0.999, 0, 0]  # overlaps [0, 1] on the same line without sharing a vertex index
    assert oracle.count_intersections(oracle.OracleScene(mesh(xs, edges=[[0, 1], [6, 7]])), xs) == 1
    # points with radius: overlapping spheres count, separated ones do not
    xp = np.array([[0.0, 0, 0], [3e-3, 0, 0], [1e-2, 0, 0]])
    r = np.array([2e-3, 2e-3, 2e-3])
    assert oracle.count_intersections(oracle.OracleScene(mesh(xp, points=[0, 1, 2], radius=r)), xp) == 1


def test_boundary_contacts_count():
    # a zero-radius point exactly on a triangle's edge, and collinear edges
    # that touch at one end point (distinct vertex indices), are intersections
    tri = np.array([[0.0, 0, 0], [1.0, 0, 0], [0, 1.0, 0], [0.5, 0.0, 0.0]])
    assert oracle.count_intersections(oracle.OracleScene(mesh(tri, tris=[[0, 1, 2]], points=[3])), tri) == 1
    x = np.array([[0.0, 0, 0], [1.0, 0, 0], [1.0, 0, 0], [2.0, 0, 0]])
    assert oracle.count_intersections(oracle.OracleScene(mesh(x, edges=[[0, 1], [2, 3]])), x) == 1
    x[2, 0] = np.nextafter(1.0, 2.0)
    assert oracle.count_intersections(oracle.OracleScene(mesh(x, edges=[[0, 1], [2, 3]])), x) == 0
