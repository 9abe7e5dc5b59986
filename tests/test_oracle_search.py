"""Pins of the oracle's proximity search (Sec. 3.1, Eq. relationship_P).

P10: the all-pairs candidate set equals the sorted-axis window candidate set
and an independent numpy brute force of the same box predicate, including
boxes exactly D apart; P is the candidates closer than D.
"""
import math
from types import SimpleNamespace as NS

import numpy as np
import pytest

import oracle
from paper_2211_04045_gb300 import scenes


def random_soup(rng, nv=40, nt=30, ne=35, npts=8, scale=0.02, radius=0.0):
    x = rng.uniform(0.0, scale, size=(nv, 3))
    tris = np.array([rng.choice(nv, 3, replace=False) for _ in range(nt)], np.int32)
    edges = np.array([rng.choice(nv, 2, replace=False) for _ in range(ne)], np.int32)
    points = rng.choice(nv, npts, replace=False).astype(np.int32)
    inv_mass = np.where(rng.uniform(size=nv) < 0.2, 0.0, 1.0)
    rad = None if radius == 0.0 else np.where(np.isin(np.arange(nv), points), radius, 0.0)
    return NS(n_verts=nv, inv_mass=inv_mass, radius=rad, tris=tris, edges=edges,
              len_edges=np.zeros((0, 2), np.int32), points=points), x


def numpy_candidates(sc, x, xt, D):
    """Independent brute force of the candidate predicate (R3, R4)."""
    n = sc.n_verts
    rho = np.zeros(n) if sc.radius is None else sc.radius
    static = (sc.inv_mass == 0) & np.all(x == xt, axis=1)
    coll = np.zeros(n, bool)
    coll[sc.tris.ravel()] = True
    coll[sc.edges.ravel()] = True
    coll[sc.points] = True
    ispt = np.zeros(n, bool)
    ispt[sc.points] = True
    vc = np.nonzero(coll)[0]

    def near(alo, ahi, blo, bhi):
        return bool(np.all(blo - ahi <= D) and np.all(alo - bhi <= D))

    out = set()
    for a in vc:
        alo, ahi = x[a] - rho[a], x[a] + rho[a]
        for t, tv in enumerate(sc.tris):
            if a in tv or (static[a] and static[tv].all()):
                continue
            if near(alo, ahi, x[tv].min(0), x[tv].max(0)):
                out.add((0 << 62) | (int(a) << 31) | t)
    E = sc.edges
    for i in range(len(E)):
        for j in range(i + 1, len(E)):
            if set(E[i]) & set(E[j]) or (static[E[i]].all() and static[E[j]].all()):
                continue
            if near(x[E[i]].min(0), x[E[i]].max(0), x[E[j]].min(0), x[E[j]].max(0)):
                out.add((1 << 62) | (i << 31) | j)
    for a in sc.points:
        for b in vc:
            if b == a or (ispt[b] and b < a) or (static[a] and static[b]):
                continue
            if near(x[a] - rho[a], x[a] + rho[a], x[b] - rho[b], x[b] + rho[b]):
                out.add((2 << 62) | (int(a) << 31) | int(b))
    return np.array(sorted(out), dtype=np.uint64)


@pytest.mark.parametrize("seed", range(16))
def test_candidates_three_ways(seed):
    rng = np.random.default_rng(seed)
    sc, x = random_soup(rng, radius=0.0 if seed % 2 else 1e-3)
    xt = x.copy()
    xt[rng.uniform(size=len(x)) < 0.5] += 1e-3
    osc = oracle.OracleScene(sc)
    D = 4e-3
    brute = oracle.candidates(osc, x, D, mode=0, x_tilde=xt)
    window = oracle.candidates(osc, x, D, mode=1, x_tilde=xt)
    ref = numpy_candidates(sc, x, xt, D)
    assert np.array_equal(brute, window)
    assert np.array_equal(brute, ref)
    keys, dist = oracle.proximity(osc, x, D, mode=1, x_tilde=xt)
    assert np.all(dist < D)
    assert set(keys.tolist()) <= set(brute.tolist())


def test_boundary_gap_exactly_D():
    # boxes exactly D apart on one axis are candidates; a hair further are not
    D = 0.5
    base = np.array([[0.0, 0, 0], [1.0, 0, 0], [0, 1.0, 0]])
    for gap, expect in ((0.5, 1), (np.nextafter(0.5, 1.0), 0)):
        x = np.concatenate([base, [[-gap, 0.25, 0.0]]])
        sc = NS(n_verts=4, inv_mass=np.ones(4), radius=None, tris=np.array([[0, 1, 2]], np.int32),
                edges=np.zeros((0, 2), np.int32), len_edges=np.zeros((0, 2), np.int32),
                points=np.array([3], np.int32))
        osc = oracle.OracleScene(sc)
        for mode in (0, 1):
            k = oracle.candidates(osc, x, D, mode=mode)
            vt = [int(q) for q in k if int(q) >> 62 == 0]
            assert len(vt) == expect
        assert np.array_equal(numpy_candidates(sc, x, x, D), oracle.candidates(osc, x, D, mode=0))


def test_window_keeps_a_gap_that_rounds_to_D():
    # the computed gap fl(lo_b - hi_a) of these operands rounds to D while the
    # window end fl(hi_a + D) lies below lo_b: the sorted-axis window must
    # widen by its slack to keep the pair that the box test (R3) accepts
    D = 4e-3
    ah, bl = -0.0025478467492858173, 0.001452153250714183
    assert bl - ah == D and bl > ah + D
    x = np.array([[ah, 1e-3, 1e-3], [bl, 0.0, 0.0], [bl + 0.01, 0.0, 2e-3], [bl + 0.005, 2e-3, 0.0]])
    sc = NS(n_verts=4, inv_mass=np.ones(4), radius=None, tris=np.array([[1, 2, 3]], np.int32),
            edges=np.zeros((0, 2), np.int32), len_edges=np.zeros((0, 2), np.int32), points=np.array([0], np.int32))
    osc = oracle.OracleScene(sc)
    k0 = oracle.candidates(osc, x, D, mode=0)
    assert (0 << 62) | (0 << 31) | 0 in [int(q) for q in k0]
    assert np.array_equal(oracle.candidates(osc, x, D, mode=1), k0)
    assert np.array_equal(numpy_candidates(sc, x, x, D), k0)


def test_window_equals_brute_on_scene():
    sc = scenes.two_cloths(n=20, side=0.2, sep=0.003, omega=6.0, noise=0.3, seed=3)
    x0, xt, _ = scenes.initial(sc)
    osc = oracle.OracleScene(sc)
    for x in (x0, xt):
        a = oracle.candidates(osc, x, 4e-3, mode=0, x_tilde=xt)
        b = oracle.candidates(osc, x, 4e-3, mode=1, x_tilde=xt)
        assert len(a) > 100 and np.array_equal(a, b)


def test_proximity_is_distance_filter():
    # P = {candidates: dist < D} with dist from the pinned distance functions
    rng = np.random.default_rng(7)
    sc, x = random_soup(rng, nv=30, nt=20, ne=25, npts=5)
    osc = oracle.OracleScene(sc)
    D = 6e-3
    cand = oracle.candidates(osc, x, D, mode=0)
    keys, dist = oracle.proximity(osc, x, D, mode=0)
    expect = []
    for k in cand.tolist():
        kind, a, b = k >> 62, (k >> 31) & 0x7FFFFFFF, k & 0x7FFFFFFF
        if kind == 0:
            d = oracle.point_triangle_dist(x[a], *x[sc.tris[b]])
        elif kind == 1:
            d = oracle.segment_segment_dist(*x[sc.edges[a]], *x[sc.edges[b]])[0]
        else:
            dv = x[a] - x[b]
            d = math.sqrt((dv[0] * dv[0] + dv[1] * dv[1]) + dv[2] * dv[2])
        if d < D:
            expect.append((k, d))
    assert keys.tolist() == [k for k, _ in expect]
    assert np.array_equal(dist, np.array([d for _, d in expect]))
