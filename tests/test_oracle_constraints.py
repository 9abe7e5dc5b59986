"""Closed-form pins of the oracle's constraints and projection (Sec. 4).

P6: a vertex h < delta above a fixed triangle, y = x: one projected
    Gauss-Seidel update lifts it to exactly delta (the volume constraint is
    linear in the vertex's height).
P7: a vertex-vertex pair at distance d < delta: one update separates it to
    rho_a + rho_b + delta.
P8: an edge stretched to 1.5 L0 with only its length constraint: one update
    gives sigma L0 along u.
"""
from types import SimpleNamespace as NS

import numpy as np
import pytest

import oracle


def mini(inv_mass, tris=(), edges=(), len_edges=(), points=(), radius=None):
    inv_mass = np.asarray(inv_mass, float)
    return NS(n_verts=len(inv_mass), inv_mass=inv_mass, radius=None if radius is None else np.asarray(radius, float),
              tris=np.asarray(tris, np.int32).reshape(-1, 3), edges=np.asarray(edges, np.int32).reshape(-1, 2),
              len_edges=np.asarray(len_edges, np.int32).reshape(-1, 2), points=np.asarray(points, np.int32))


@pytest.mark.parametrize("h", [0.1e-3, 0.4e-3, 0.9e-3])
@pytest.mark.parametrize("flip", [False, True])
@pytest.mark.parametrize("below", [False, True])
def test_p6_vertex_triangle_lift(h, flip, below):
    tri = np.array([[0.0, 0, 0], [1e-2, 0, 0], [0, 1e-2, 0]])
    z = -h if below else h
    x = np.concatenate([[[2e-3, 3e-3, z]], tri])
    t = [[1, 3, 2]] if flip else [[1, 2, 3]]
    sc = mini([2.0, 0, 0, 0], tris=t, points=[0])
    delta = 1e-3
    y = oracle.backward_once(oracle.OracleScene(sc), oracle.params(delta=delta), x, x, x)
    target = -delta if below else delta
    assert abs(y[0, 2] - target) <= 1e-15
    assert np.all(y[0, :2] == x[0, :2])
    assert np.array_equal(y[1:], x[1:])


def test_vt_interior_value_and_gradient():
    # interior closest point: c = h/delta - 1; vertex gradient along +n / delta;
    # triangle gradients along -n weighted by the barycentric coordinates
    delta = 1e-3
    h = 0.3e-3
    p = np.array([[0.2e-2, 0.3e-2, h], [0, 0, 0], [1e-2, 0, 0], [0, 1e-2, 0]])
    ok, c0, g = oracle.contact_constraint(oracle.VT, p, [0.0], delta)
    assert ok
    assert abs(c0 - (h / delta - 1.0)) < 1e-12
    assert np.allclose(g[0], [0, 0, 1.0 / delta], rtol=1e-12, atol=1e-9)
    bary = np.array([1 - 0.2 - 0.3, 0.2, 0.3])
    for k in range(3):
        assert np.isclose(g[1 + k, 2], -bary[k] / delta, rtol=1e-9)
    assert np.allclose(g.sum(axis=0), 0.0, atol=1e-9)
    # in-plane terms of the triangle gradients (area change) scale with h
    p2 = p.copy()
    p2[0, 2] = h / 2
    _, _, g2 = oracle.contact_constraint(oracle.VT, p2, [0.0], delta)
    assert np.allclose(g2[1:, :2], 0.5 * g[1:, :2], rtol=1e-9, atol=1e-9)


def test_ee_crossing_value():
    # crossing edges at distance d: c = d/delta - 1 and the gradients push the
    # edges apart along the common normal
    delta = 1e-3
    d = 0.25e-3
    p = np.array([[-1e-2, 0, d], [1e-2, 0, d], [0, -1e-2, 0], [0, 1e-2, 0]])
    ok, c0, g = oracle.contact_constraint(oracle.EE, p, [0.0, 0.0], delta)
    assert ok
    assert abs(c0 - (d / delta - 1.0)) < 1e-12
    assert g[0, 2] > 0 and g[1, 2] > 0 and g[2, 2] < 0 and g[3, 2] < 0
    assert np.allclose(g.sum(axis=0), 0.0, atol=1e-9)


def test_ee_parallel_gap_form():
    delta = 1e-3
    d = 0.5e-3
    p = np.array([[0.0, 0, d], [1e-2, 0, d], [0.25e-2, 0, 0], [1.25e-2, 0, 0]])
    ok, c0, g = oracle.contact_constraint(oracle.EE, p, [0.0, 0.0], delta)
    assert ok
    assert abs(c0 - (d / delta - 1.0)) < 1e-12
    # weights (1-s, s) and -(1-t), -t along +z with 1/delta
    assert np.allclose(g[:, :2], 0.0)
    assert np.isclose(g[0, 2] + g[1, 2], 1.0 / delta)
    assert np.isclose(g[2, 2] + g[3, 2], -1.0 / delta)


@pytest.mark.parametrize("sin_theta,gap_form", [(1e-7, True), (1e-5, False)])
def test_ee_near_parallel_threshold(sin_theta, gap_form):
    # R7: edges with sin(theta) below 1e-6 take the gap form, gradient
    # (1-s, s, -(1-t), -t) n / delta; above it the volume form, whose gradient
    # over the tiny reference volume of near-parallel edges is far larger.
    # Both give c = d/delta - 1 here (the edges lie in parallel planes).
    delta, d = 1e-3, 0.5e-3
    p = np.array([[0.0, 0, d], [1e-2, 0, d], [0.2e-2, 0, 0], [0.8e-2, 0.6e-2 * sin_theta, 0]])
    ok, c0, g = oracle.contact_constraint(oracle.EE, p, [0.0, 0.0], delta)
    dist, s, t = oracle.segment_segment_dist(*p)
    assert ok and abs(c0 - (dist / delta - 1.0)) < 1e-12
    gap_g = np.outer([1.0 - s, s, -(1.0 - t), -t], [0.0, 0.0, 1.0]) / delta
    assert np.array_equal(g, gap_g) == gap_form
    if not gap_form:
        assert np.abs(g).max() > 1e3 / delta


@pytest.mark.parametrize("radius", [0.0, 2e-3])
def test_p7_vertex_vertex_separation(radius):
    delta = 1e-3
    R = 2 * radius + delta
    d = 0.4 * R
    u = np.array([1.0, 2.0, 2.0]) / 3.0
    x = np.array([[0.1, 0.2, 0.3], [0.1, 0.2, 0.3]]) + np.array([[0, 0, 0], d * u])
    sc = mini([1.0, 1.0], points=[0, 1], radius=[radius, radius])
    y = oracle.backward_once(oracle.OracleScene(sc), oracle.params(delta=delta), x, x, x)
    sep = np.linalg.norm(y[1] - y[0])
    assert abs(sep - R) <= 1e-14
    assert np.allclose(np.cross(y[1] - y[0], u), 0.0, atol=1e-15)
    assert np.allclose(0.5 * (y[0] + y[1]), 0.5 * (x[0] + x[1]), atol=1e-16)


@pytest.mark.parametrize("sigma", [1.0, 1.1, 1.3])
def test_p8_edge_length(sigma):
    u = np.array([0.6, 0.0, 0.8])
    L0 = 0.02
    y0 = np.array([[0.0, 0.0, 0.0], L0 * u])
    y = np.array([[0.0, 0.0, 0.0], 1.5 * L0 * u])
    sc = mini([1.0, 3.0], len_edges=[[0, 1]])
    out = oracle.backward_once(oracle.OracleScene(sc), oracle.params(sigma=sigma), y0, y, y0)
    d = out[1] - out[0]
    assert abs(np.linalg.norm(d) - sigma * L0) <= 1e-15
    assert np.allclose(np.cross(d, u), 0.0, atol=1e-16)
    # inverse-mass weighted: the heavier vertex moves a third as much
    m0 = np.linalg.norm(out[0] - y[0])
    m1 = np.linalg.norm(out[1] - y[1])
    assert abs(m1 - 3.0 * m0) <= 1e-15


def test_edge_not_active_below_sigma():
    u = np.array([0.0, 1.0, 0.0])
    y0 = np.array([[0.0, 0, 0], 0.02 * u])
    y = np.array([[0.0, 0, 0], 0.021 * u])  # 1.05 L0 < 1.1 L0
    sc = mini([1.0, 1.0], len_edges=[[0, 1]])
    out = oracle.backward_once(oracle.OracleScene(sc), oracle.params(), y0, y, y0)
    assert np.array_equal(out, y)
