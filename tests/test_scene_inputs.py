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
