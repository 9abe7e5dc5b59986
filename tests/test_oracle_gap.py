"""Pins of the gap-constraint variant (the comparison constraints of the gap
figure in Sec. 4.1): c = d/delta - 1 with gradient w_v n / delta.

* A vertex above a fixed triangle, and two crossing edges, reach distance
  exactly delta after one projected update (the gap is linear along n).
* The gradient equals the derivative of the distance (finite differences of
  the oracle's own distance functions, away from the kinks).
* The form parameter reaches the step: gap and volume give different y when
  the triangle's vertices move too.
"""
from types import SimpleNamespace as NS

import numpy as np
import pytest

import oracle


def mini(inv_mass, tris=(), edges=(), points=()):
    inv_mass = np.asarray(inv_mass, float)
    return NS(n_verts=len(inv_mass), inv_mass=inv_mass, radius=None, tris=np.asarray(tris, np.int32).reshape(-1, 3),
              edges=np.asarray(edges, np.int32).reshape(-1, 2), len_edges=np.zeros((0, 2), np.int32),
              points=np.asarray(points, np.int32))


@pytest.mark.parametrize("h", [0.1e-3, 0.5e-3, 0.9e-3])
def test_vertex_lift_to_delta(h):
    tri = np.array([[0.0, 0, 0], [1e-2, 0, 0], [0, 1e-2, 0]])
    x = np.vstack([[[2e-3, 3e-3, h]], tri])
    sc = mini([1.5, 0, 0, 0], tris=[[1, 2, 3]], points=[0])
    y = oracle.backward_once(oracle.OracleScene(sc), oracle.params(constraint_form=1), x, x, x)
    assert abs(y[0, 2] - 1e-3) <= 1e-15
    assert np.all(y[0, :2] == x[0, :2]) and np.array_equal(y[1:], x[1:])


@pytest.mark.parametrize("h", [0.2e-3, 0.6e-3])
def test_crossing_edges_separate_to_delta(h):
    x = np.array([[-5e-3, 0, h], [5e-3, 0, h], [0, -5e-3, 0], [0, 5e-3, 0]])
    sc = mini([1.0, 1.0, 1.0, 1.0], edges=[[0, 1], [2, 3]])
    y = oracle.backward_once(oracle.OracleScene(sc), oracle.params(constraint_form=1), x, x, x)
    # each edge moves half of delta - h along z; the distance becomes delta
    assert np.allclose(y[:2, 2], h + 0.5 * (1e-3 - h), atol=1e-16, rtol=0)
    assert np.allclose(y[2:, 2], -0.5 * (1e-3 - h), atol=1e-16, rtol=0)
    assert np.array_equal(y[:, :2], x[:, :2])


def numeric_grad(f, p, eps=1e-9):
    g = np.zeros_like(p)
    for i in range(p.shape[0]):
        for k in range(3):
            a, b = p.copy(), p.copy()
            a[i, k] += eps
            b[i, k] -= eps
            g[i, k] = (f(a) - f(b)) / (2 * eps)
    return g


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("region", ["inside", "edge"])
def test_vt_gradient_is_distance_derivative(seed, region):
    rng = np.random.default_rng(seed)
    tri = rng.normal(0, 5e-3, size=(3, 3))
    w = rng.dirichlet([2, 2, 2]) if region == "inside" else np.array([0.5 + 0.3 * rng.uniform(-1, 1), 0.0, 0.0])
    if region == "edge":
        w[1] = 1.0 - w[0]
    foot = w @ tri
    nrm = np.cross(tri[1] - tri[0], tri[2] - tri[0])
    nrm /= np.linalg.norm(nrm)
    out = np.zeros(3)
    if region == "edge":  # push outward across edge (0,1) within the plane, then up
        e = tri[1] - tri[0]
        out = np.cross(nrm, e)
        out /= np.linalg.norm(out)
        if np.dot(out, tri[2] - foot) > 0:
            out = -out
    p0 = foot + 4e-4 * nrm + 3e-4 * out
    pos = np.vstack([p0, tri])
    delta = 1e-3
    ok, c0, g = oracle.contact_constraint(oracle.VT, pos, [0.0], delta, form=1)
    assert ok
    d = oracle.point_triangle_dist(*pos)
    assert abs(c0 - (d / delta - 1.0)) <= 1e-15
    gn = numeric_grad(lambda q: oracle.point_triangle_dist(*q) / delta, pos)
    assert np.max(np.abs(g - gn)) <= 1e-5 * np.max(np.abs(gn))


@pytest.mark.parametrize("seed", range(6))
def test_ee_gradient_is_distance_derivative(seed):
    rng = np.random.default_rng(100 + seed)
    a, b = rng.normal(0, 5e-3, 3), rng.normal(0, 5e-3, 3)
    s, t = rng.uniform(0.2, 0.8, 2)
    m = a + s * (b - a)
    u = rng.normal(size=3)
    u -= np.dot(u, b - a) / np.dot(b - a, b - a) * (b - a)
    u /= np.linalg.norm(u)
    v = np.cross(b - a, u)
    v /= np.linalg.norm(v)
    q = m + 3e-4 * u                          # closest point of the second edge
    c = q - t * 6e-3 * v
    d = q + (1 - t) * 6e-3 * v
    pos = np.vstack([a, b, c, d])
    delta = 1e-3
    ok, c0, g = oracle.contact_constraint(oracle.EE, pos, [0.0, 0.0], delta, form=1)
    assert ok
    dist = oracle.segment_segment_dist(*pos)[0]
    assert abs(c0 - (dist / delta - 1.0)) <= 1e-15
    gn = numeric_grad(lambda qq: oracle.segment_segment_dist(*qq)[0] / delta, pos)
    assert np.max(np.abs(g - gn)) <= 1e-5 * np.max(np.abs(gn))


def test_form_reaches_the_step():
    tri = np.array([[0.0, 0, 0], [1e-2, 0, 0], [0, 1e-2, 0]])
    x = np.vstack([[[2e-3, 3e-3, 0.4e-3]], tri])
    sc = mini([1.0, 1.0, 1.0, 1.0], tris=[[1, 2, 3]], points=[0])
    osc = oracle.OracleScene(sc)
    yv = oracle.backward_once(osc, oracle.params(constraint_form=0), x, x, x)
    yg = oracle.backward_once(osc, oracle.params(constraint_form=1), x, x, x)
    assert not np.array_equal(yv, yg)
    # the gap form separates the vertex from its closest point by exactly delta along the normal
    wts = np.array([1 - 0.2 - 0.3, 0.2, 0.3])
    assert abs((yg[0, 2] - wts @ yg[1:, 2]) - 1e-3) <= 1e-15
