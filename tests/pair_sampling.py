"""Sampled check of a proximity set P at sizes where the oracle's whole-scene
search is too slow: for sampled query primitives, their pairs in P are
recomputed one by one with the oracle's distance routines over every
primitive whose box passes the candidate test (R3: on every axis the
rounded gap is at most D), with the exclusions of R4 (shared vertex; every
vertex static) and the distances of R5 (vertex-triangle minus the vertex's
radius, segment-segment, centre distance minus both radii; a point pair
once, keyed by its lower id).  Test infrastructure (imports the oracle)."""
import numpy as np

import oracle

VT, EE, VV = 0, 1, 2


def jittered(sc, x0, sigma, seed):
    rng = np.random.default_rng(seed)
    x = x0.copy()
    mov = sc.inv_mass > 0
    x[mov] += rng.normal(0.0, sigma, size=(int(mov.sum()), 3))
    return x


def _key(kind, a, b):
    return (kind << 62) | (int(a) << 31) | int(b)


def check_sampled_pairs(sc, x, xt, D, got, n, seed):
    """Asserts that got (key -> distance) holds exactly the pairs of P of n
    sampled collision vertices (VT), n edges (EE) and n points (VV); returns
    the number of pairs checked."""
    rng = np.random.default_rng(seed)
    rho = sc.radius if sc.radius is not None else np.zeros(len(x))
    static = (sc.inv_mass == 0) & np.all(x == xt, axis=1)
    tris, edges, pts = sc.tris, sc.edges, np.asarray(sc.points, dtype=np.int64)
    is_point = np.zeros(len(x), bool)
    is_point[pts] = True
    coll = np.zeros(len(x), bool)
    coll[tris.ravel()] = True
    coll[edges.ravel()] = True
    coll[pts] = True
    vc = np.nonzero(coll)[0]
    by_id = {}
    for k, d in got.items():
        kind, a, b = k >> 62, (k >> 31) & 0x7FFFFFFF, k & 0x7FFFFFFF
        by_id.setdefault((kind, a), {})[k] = d
        if kind != VT:
            by_id.setdefault((kind, b), {})[k] = d

    def near(alo, ahi, blo, bhi):
        return np.all((blo - ahi <= D) & (alo - bhi <= D), axis=1)

    tlo, thi = x[tris].min(axis=1), x[tris].max(axis=1)
    elo, ehi = x[edges].min(axis=1), x[edges].max(axis=1)
    vlo, vhi = x[vc] - rho[vc, None], x[vc] + rho[vc, None]
    checked = 0
    for a in rng.choice(vc, min(n, len(vc)), replace=False):
        want = {}
        for t in np.nonzero(near(x[a] - rho[a], x[a] + rho[a], tlo, thi))[0]:
            tv = tris[t]
            if a in tv or (static[a] and static[tv].all()):
                continue
            d = oracle.point_triangle_dist(x[a], *x[tv]) - rho[a]
            if d < D:
                want[_key(VT, a, t)] = d
        assert by_id.get((VT, int(a)), {}) == want, ("VT", int(a))
        checked += len(want)
    for e in rng.choice(len(edges), min(n, len(edges)), replace=False):
        want = {}
        for f in np.nonzero(near(elo[e], ehi[e], elo, ehi))[0]:
            if f == e or np.intersect1d(edges[e], edges[f]).size or static[np.r_[edges[e], edges[f]]].all():
                continue
            d = oracle.segment_segment_dist(*x[edges[e]], *x[edges[f]])[0]
            if d < D:
                want[_key(EE, min(e, f), max(e, f))] = d
        assert by_id.get((EE, int(e)), {}) == want, ("EE", int(e))
        checked += len(want)
    for p in rng.choice(pts, min(n, len(pts)), replace=False):
        want = {}
        for j in np.nonzero(near(x[p] - rho[p], x[p] + rho[p], vlo, vhi))[0]:
            w = vc[j]
            if w == p or (static[p] and static[w]):
                continue
            a, b = (p, w) if not is_point[w] else (min(p, w), max(p, w))
            d = (np.linalg.norm(x[a] - x[b]) - rho[a]) - rho[b]
            if d < D:
                want[_key(VV, a, b)] = d
        have = by_id.get((VV, int(p)), {})
        assert set(have) == set(want), ("VV", int(p))
        for k in want:
            assert abs(have[k] - want[k]) <= 1e-15, ("VV", int(p), k)
        checked += len(want)
    return checked
