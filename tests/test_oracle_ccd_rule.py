"""Pins of the CCD-based step size (the comparison scheme of Sec. 5.1) and of
the CCD safety check, in the oracle (no GPU).

Under the CCD rule every vertex's step is capped by the global bound
0.5 gamma D^(l) instead of its own 0.5 gamma D_i, and the CCD of each pair's
segment decides the rest: a hit at time t scales the step of the pair's
vertices by t/2, the segments are tested again, and after ccd_rounds rounds a
remaining hit keeps the scene where it is for the iteration."""
from types import SimpleNamespace as NS

import numpy as np
import pytest

import oracle
from paper_2211_04045_gb300 import scenes

from test_oracle_step import colliding_cases, free_cloth


def vertex_over_triangle(h):
    """A fixed triangle in the plane z = 0 and a free vertex at height h over
    its interior."""
    x = np.array([[-0.1, -0.1, 0.0], [0.1, -0.1, 0.0], [0.0, 0.1, 0.0], [0.0, 0.0, h]])
    sc = NS(n_verts=4, inv_mass=np.array([0.0, 0.0, 0.0, 1.0]), radius=None,
            tris=np.array([[0, 1, 2]], np.int32), edges=np.zeros((0, 2), np.int32),
            len_edges=np.zeros((0, 2), np.int32), points=np.array([3], np.int32))
    return sc, x


def test_no_pairs_in_reach_the_rules_coincide():
    # with no pair within D^max every D_i equals D^(l): both rules take the
    # same steps and the CCD finds nothing
    sc = free_cloth()
    x0 = sc.x0
    xt = x0 + np.array([0.03, -0.04, 0.0])
    osc = oracle.OracleScene(sc)
    a, sa, _ = oracle.handle_step(osc, oracle.params(), x0, xt)
    b, sb, _ = oracle.handle_step(osc, oracle.params(step_rule=1), x0, xt)
    assert np.array_equal(a, b) and sa == sb and sb["ccd_clamps"] == 0


def test_clamped_vertex_moves_halfway_to_the_plane():
    # h = 1.5 mm, target 1.5 mm below the plane (|dx| = 3 mm), one iteration.
    # Distance rule: alpha = 0.45 * 1.5 / 3, the vertex moves 0.675 mm.
    # CCD rule: the cap 0.45 D^max = 1.8 mm would cross the plane at
    # t = 1.5 / 1.8; the step is scaled by t/2, so the vertex stops at h/2.
    h = 1.5e-3
    sc, x = vertex_over_triangle(h)
    xt = x.copy()
    xt[3, 2] = -h
    osc = oracle.OracleScene(sc)
    d, sd, _ = oracle.handle_step(osc, oracle.params(max_iters=0), x, xt)
    assert abs(d[3, 2] - (h - 0.45 * h)) < 1e-15 and sd["ccd_clamps"] == 0
    c, st, _ = oracle.handle_step(osc, oracle.params(max_iters=0, step_rule=1), x, xt)
    assert abs(c[3, 2] - 0.5 * h) < 1e-15
    assert np.array_equal(c[:3], x[:3]) and c[3, 0] == 0.0 and c[3, 1] == 0.0
    assert st["ccd_clamps"] == 1 and st["iterations"] == 1 and st["converged"] == 0


def test_no_rounds_left_freezes_the_step():
    # ccd_rounds = 0: the first hit keeps every vertex where it is
    h = 1.5e-3
    sc, x = vertex_over_triangle(h)
    xt = x.copy()
    xt[3, 2] = -h
    c, st, _ = oracle.handle_step(oracle.OracleScene(sc), oracle.params(max_iters=0, step_rule=1, ccd_rounds=0),
                                  x, xt)
    assert np.array_equal(c, x) and st["ccd_clamps"] == 1 and st["final_r_inf"] == 1.0


def test_falling_vertex_settles_above_the_plane():
    h = 1.5e-3
    sc, x = vertex_over_triangle(h)
    xt = x.copy()
    xt[3, 2] = -0.05
    osc = oracle.OracleScene(sc)
    for rule in (0, 1):
        c, st, _ = oracle.handle_step(osc, oracle.params(max_iters=400, step_rule=rule), x, xt)
        assert oracle.count_intersections(osc, c) == 0
        assert c[3, 2] > 0.0 and np.array_equal(c[:3], x[:3])


@pytest.mark.parametrize("case", range(3))
def test_ccd_rule_safety_invariants(case):
    name, sc = colliding_cases()[case]
    osc = oracle.OracleScene(sc)
    prm = oracle.params_for(sc, max_iters=120, step_rule=1)
    x, xt, _ = scenes.initial(sc)
    cap_p = 20000
    xn, st, tr = oracle.handle_step(osc, prm, x, xt, trace_iters=prm.max_iters + 2, trace_pairs=cap_p)
    for l in range(st["iterations"]):
        xl, xl1, Dl = tr["x"][l], tr["x"][l + 1], tr["Dl"][l]
        mv = np.linalg.norm(xl1 - xl, axis=1)
        # the global cap, and P holds every pair closer than D^(l)
        assert np.all(mv <= 0.5 * prm.gamma * Dl * (1 + 1e-12)), (name, l)
        held = set(tr["pair_keys"][l][:tr["n_pairs"][l]].tolist())
        fresh, _ = oracle.proximity(osc, xl, Dl, mode=0, x_tilde=xt)
        assert set(fresh.tolist()) <= held, (name, l)
        if l % 5 == 0:
            near, _ = oracle.proximity(osc, xl, 2.0 * Dl, mode=0, x_tilde=xt)
            for k in near.tolist():
                kind, a, b = k >> 62, (k >> 31) & 0x7FFFFFFF, k & 0x7FFFFFFF
                vs = [a, *sc.tris[b]] if kind == 0 else ([*sc.edges[a], *sc.edges[b]] if kind == 1 else [a, b])
                rho = None if kind != 2 or sc.radius is None else sc.radius[vs]
                hit, _ = oracle.ccd(kind, xl[vs], xl1[vs], rho)
                assert not hit, (name, l, k)
    assert oracle.count_intersections(osc, xn) == 0


@pytest.mark.parametrize("case", range(3))
def test_safety_check_finds_nothing_under_the_distance_rule(case):
    # the distance rule is safe by construction (Sec. 5): the CCD check adds
    # no clamp and changes nothing
    name, sc = colliding_cases()[case]
    osc = oracle.OracleScene(sc)
    x, xt, _ = scenes.initial(sc)
    a, sa, _ = oracle.handle_step(osc, oracle.params_for(sc, max_iters=120), x, xt)
    b, sb, _ = oracle.handle_step(osc, oracle.params_for(sc, max_iters=120, ccd_check=1), x, xt)
    assert np.array_equal(a, b) and sa == sb and sb["ccd_clamps"] == 0


@pytest.mark.parametrize("case", range(3))
def test_distance_rule_segments_certified_apart(case):
    # Sec. 5's guarantee checked with the conservative CCD (not the
    # root-finding one): under the distance rule each vertex moves at most
    # 0.45 D_i per iteration, so a pair at distance d stays at least 0.1 d
    # apart along the whole segment x^(l) -> x^(l+1); 0.05 d is certified
    name, sc = colliding_cases()[case]
    osc = oracle.OracleScene(sc)
    prm = oracle.params_for(sc, max_iters=120)
    x, xt, _ = scenes.initial(sc)
    xn, st, tr = oracle.handle_step(osc, prm, x, xt, trace_iters=prm.max_iters + 2)
    checked = 0
    for l in range(0, st["iterations"], 3):
        xl, xl1, Dl = tr["x"][l], tr["x"][l + 1], tr["Dl"][l]
        near, dist = oracle.proximity(osc, xl, 2.0 * Dl, mode=0, x_tilde=xt)
        for k, d in zip(near.tolist(), dist.tolist()):
            if d < 1e-10:
                continue  # held by the D_i floor: its vertices do not move
            kind, a, b = k >> 62, (k >> 31) & 0x7FFFFFFF, k & 0x7FFFFFFF
            vs = [a, *sc.tris[b]] if kind == 0 else ([*sc.edges[a], *sc.edges[b]] if kind == 1 else [a, b])
            rho = None if kind != 2 or sc.radius is None else sc.radius[vs]
            assert not oracle.ccd_conservative(kind, xl[vs], xl1[vs], rho, tol=0.05 * d), (name, l, k, d)
            checked += 1
    assert checked > 100


def test_floor_keeps_collapsed_pairs_still_under_the_ccd_rule():
    # a 32 x 32 cloth falling onto a subdivision-3 sphere, three chain steps of
    # 2,049 iterations under the CCD-based rule: the rule collapses some pairs
    # to about 1e-17 m, where the root-finding CCD no longer sees a crossing;
    # with the R2b floor on each vertex's own D_i those vertices stay, and
    # every step ends intersection-free under the exact test
    torch = pytest.importorskip("torch")
    sc = scenes.cloth_over_sphere(n=32)
    osc = oracle.OracleScene(sc)
    prm = oracle.params_for(sc, step_rule=1)
    dyn = scenes.TorchDynamics(sc, "cpu")
    x, xt, _ = scenes.initial(sc)
    frozen = 0
    for _ in range(3):
        xn, st, _ = oracle.handle_step(osc, prm, x, xt)
        assert oracle.count_intersections(osc, xn) == 0
        frozen += st["frozen_vertices"]
        v = dyn.next_velocity(torch.tensor(xn), torch.tensor(x)).numpy()
        x, xt = xn, dyn.predict(torch.tensor(xn), torch.tensor(v)).numpy()
    assert frozen > 0  # the floor did hold vertices
