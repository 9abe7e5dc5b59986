"""Pins of the oracle's geometry against brute force, closed forms and exact
rational arithmetic (no GPU).

* distances (the dist() of Eq. relationship_P and Sec. 5) against dense
  sampling of the simplices, with the sampling error bounded;
* the signed volume of Eq. volume_by_det vanishing exactly at coplanarity;
* the exact orientation predicate against Python fractions.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle


def sample_tri(a, b, c, m):
    i, j = np.meshgrid(np.arange(m + 1), np.arange(m + 1), indexing="ij")
    keep = i + j <= m
    u, v = (i[keep] / m)[:, None], (j[keep] / m)[:, None]
    return a + u * (b - a) + v * (c - a)


def sample_seg(a, b, m):
    t = (np.arange(m + 1) / m)[:, None]
    return a + t * (b - a)


@pytest.mark.parametrize("seed", range(40))
def test_point_triangle_vs_sampling(seed):
    rng = np.random.default_rng(seed)
    a, b, c = rng.normal(size=(3, 3))
    p = rng.normal(size=3) * (0.2 + rng.uniform() * 1.5)
    m = 300
    pts = sample_tri(a, b, c, m)
    smin = np.min(np.linalg.norm(pts - p, axis=1))
    L = max(np.linalg.norm(b - a), np.linalg.norm(c - a), np.linalg.norm(c - b))
    d = oracle.point_triangle_dist(p, a, b, c)
    assert d <= smin + 1e-12
    assert d >= smin - 2.0 * L / m - 1e-12


@pytest.mark.parametrize("seed", range(40))
def test_segment_segment_vs_sampling(seed):
    rng = np.random.default_rng(100 + seed)
    a, b, c, d = rng.normal(size=(4, 3))
    if seed % 4 == 0:  # near-parallel case
        d = c + (b - a) * 0.7 + rng.normal(size=3) * 1e-9
    m = 400
    P = sample_seg(a, b, m)
    Q = sample_seg(c, d, m)
    smin = np.min(np.linalg.norm(P[:, None, :] - Q[None, :, :], axis=2))
    L = max(np.linalg.norm(b - a), np.linalg.norm(d - c))
    dist, s, t = oracle.segment_segment_dist(a, b, c, d)
    assert dist <= smin + 1e-12
    assert dist >= smin - 2.0 * L / m - 1e-12
    # the returned parameters realise the distance
    pp = a + s * (b - a)
    qq = c + t * (d - c)
    assert 0.0 <= s <= 1.0 and 0.0 <= t <= 1.0
    assert abs(np.linalg.norm(pp - qq) - dist) <= 1e-12 * (1.0 + dist)


def test_distance_closed_forms():
    a, b, c = np.array([0.0, 0, 0]), np.array([1.0, 0, 0]), np.array([0.0, 1, 0])
    # above the interior: the height
    assert oracle.point_triangle_dist([0.25, 0.25, 0.375], a, b, c) == 0.375
    # beyond a vertex: distance to the vertex
    assert oracle.point_triangle_dist([-3.0, -4.0, 0.0], a, b, c) == 5.0
    # beyond an edge, in plane
    assert oracle.point_triangle_dist([0.5, -0.75, 0.0], a, b, c) == 0.75
    # crossing segments at right angles, offset h
    d, s, t = oracle.segment_segment_dist([-1.0, 0, 0.5], [1.0, 0, 0.5], [0, -1.0, 0], [0, 1.0, 0])
    assert d == 0.5 and s == 0.5 and t == 0.5
    # parallel overlapping segments
    d, s, t = oracle.segment_segment_dist([0.0, 0, 0], [2.0, 0, 0], [1.0, 0.25, 0], [3.0, 0.25, 0])
    assert d == 0.25
    # collinear, disjoint: the gap
    d, s, t = oracle.segment_segment_dist([0.0, 0, 0], [1.0, 0, 0], [1.5, 0, 0], [3.0, 0, 0])
    assert d == 0.5 and s == 1.0 and t == 0.0
    # point-segment clamps
    d, t = oracle.point_segment_dist([2.0, 1.0, 0.0], [0.0, 0, 0], [1.0, 0, 0])
    assert t == 1.0 and d == np.sqrt(2.0)


def frac_orient(a, b, c, d):
    A = [Fraction(v) for v in a]
    B = [Fraction(v) - A[i] for i, v in enumerate(b)]
    Cc = [Fraction(v) - A[i] for i, v in enumerate(c)]
    D = [Fraction(v) - A[i] for i, v in enumerate(d)]
    det = (B[0] * (Cc[1] * D[2] - Cc[2] * D[1]) - B[1] * (Cc[0] * D[2] - Cc[2] * D[0]) +
           B[2] * (Cc[0] * D[1] - Cc[1] * D[0]))
    return (det > 0) - (det < 0)


@pytest.mark.parametrize("seed", range(30))
def test_signed_volume_zero_at_coplanarity(seed):
    # P1: integer points on one plane give an exactly zero FP64 volume, for
    # every assignment of the four points
    rng = np.random.default_rng(seed)
    a, b, c = rng.integers(-50, 50, size=(3, 3)).astype(float)
    i, j = rng.integers(-5, 6, size=2)
    d = a + i * (b - a) + j * (c - a)
    for q in ([a, b, c, d], [d, a, b, c], [b, d, a, c], [c, b, d, a]):
        assert oracle.signed_volume(*q) == 0.0
        assert oracle.orient3d_exact(*q) == 0
    # off the plane by one unit: nonzero, sign as the rational determinant
    e = d + np.cross(b - a, c - a) / max(1.0, np.abs(np.cross(b - a, c - a)).max())
    e = np.round(e)
    v = oracle.signed_volume(a, b, c, e)
    assert np.sign(v) == frac_orient(a, b, c, e)


@pytest.mark.parametrize("seed", range(60))
def test_orient3d_exact_vs_fractions(seed):
    rng = np.random.default_rng(1000 + seed)
    a, b, c = rng.normal(size=(3, 3))
    u, v = rng.normal(size=2)
    d = a + u * (b - a) + v * (c - a)  # nearly coplanar after rounding
    k = seed % 3
    if k == 1:
        d = np.nextafter(d, d + 1.0)
    elif k == 2:
        d = d + rng.normal(size=3) * 1e-14
    assert oracle.orient3d_exact(a, b, c, d) == frac_orient(a, b, c, d)
    f = rng.normal(size=3)
    assert oracle.orient3d_exact(a, b, c, f) == frac_orient(a, b, c, f)
