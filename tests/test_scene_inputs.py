"""The method assumes an intersection-free start (x^t in Omega, Sec. 3):
every workload generator's initial state passes the oracle's exact
intersection count, at full size where that count finishes in seconds and
at reduced size otherwise (same geometry), and the seeded generators are
reproducible (no GPU)."""
import numpy as np
import pytest

import oracle
from paper_2211_04045_gb300 import scenes as S

CASES = {
    "cloth_sphere (full)": lambda: S.cloth_over_sphere(),
    "two_cloths (64x64, full geometry)": lambda: S.two_cloths(n=64),
    "tets (full)": lambda: S.tet_bodies(),
    "knot (24 x 81)": lambda: S.tube_knot(around=24, rings=81),
    "hair_sand (400 strands, 2000 grains)": lambda: S.hair_sand(n_strands=400, segs=16, n_points=2000),
    "normal_flow (full)": lambda: S.normal_flow_torus(),
    "normal_flow grow": lambda: S.normal_flow_torus(n_major=48, n_minor=16, R=0.015, r=0.01, sign=1.0),
    "rotating_sphere (full)": lambda: S.cloth_on_rotating_sphere(),
}


@pytest.mark.parametrize("name", list(CASES))
def test_initial_state_is_intersection_free(name):
    sc = CASES[name]()
    assert oracle.count_intersections(oracle.OracleScene(sc), sc.x0) == 0


def test_generators_are_seeded():
    a, b = S.two_cloths(n=32, seed=5), S.two_cloths(n=32, seed=5)
    assert np.array_equal(S.initial(a)[1], S.initial(b)[1])
    c = S.two_cloths(n=32, seed=6)
    assert not np.array_equal(S.initial(a)[1], S.initial(c)[1])


def test_serving_requests_are_smooth_small_steps():
    # the serving stream's targets: a smooth field of at most 1 mm that moves
    # no fixed vertex, reproducible from its seed; on the small tube pair,
    # with the scene's own parameters, such a request converges in a few
    # oracle iterations and stays intersection-free
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    sc = S.tube_knot(around=16, rings=65, r=0.004, helix_r=0.0055, pitch=0.03, ring_dz=0.002)
    d1 = bench.smooth_displacement(sc, np.random.default_rng(3))
    d2 = bench.smooth_displacement(sc, np.random.default_rng(3))
    assert np.array_equal(d1, d2)
    assert np.abs(d1).max() <= 1e-3 and np.abs(d1).max() > 0.0
    assert not np.any(d1[sc.inv_mass == 0.0])
    # neighbouring vertices move alike: each component is a sinusoid of
    # amplitude at most 1 mm and wavelength at least a third of the extent,
    # so along an edge between movable vertices it changes by at most
    # 1 mm * 2 pi * 3 / extent * edge length
    e = np.asarray(sc.edges)
    e = e[(sc.inv_mass[e[:, 0]] > 0.0) & (sc.inv_mass[e[:, 1]] > 0.0)]
    ext = float(np.ptp(sc.x0, axis=0).max())
    length = np.linalg.norm(sc.x0[e[:, 0]] - sc.x0[e[:, 1]], axis=1)
    assert np.all(np.abs(d1[e[:, 0]] - d1[e[:, 1]]).max(axis=1) <= 1e-3 * 2 * np.pi * 3 / ext * length * (1 + 1e-9))
    osc = oracle.OracleScene(sc)
    xn, st, _ = oracle.handle_step(osc, oracle.params_for(sc), sc.x0, sc.x0 + d1)
    assert st["converged"] == 1 and st["iterations"] < 64
    assert oracle.count_intersections(osc, xn) == 0
