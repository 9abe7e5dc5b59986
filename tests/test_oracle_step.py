"""Pins of the oracle's Algorithm 1 (no GPU).

P3: with no active constraint the forward step walks straight to the target,
    and the termination metric is the remaining fraction of the way
    (Eq. forward2); the iteration count follows from the move bound
    0.5 gamma D^max per iteration.
P4: moves below 0.45 D^max with no pair closer than D^max: one iteration and
    x^{t+1} == x~ bitwise.
P4b (R2c): a vertex whose target is not finite keeps its position exactly
    while the others reach theirs; the step never converges (r of that
    vertex stays 1) and stops after L + 1 iterations.
P5: safety of every forward step (|dx_i| < D_i/2, Sec. 5), the reuse bound of
    Eq. relationship_P (P contains every pair closer than D^(l)), no CCD hit
    on any segment of the path, and an intersection-free result.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2211_04045_gb300 import scenes


def free_cloth(n=10, spacing=0.02):
    return scenes.two_cloths(n=n, side=spacing * (n - 1), sep=0.5, omega=0.0, noise=0.0)


def test_p3_straight_walk_and_r():
    sc = free_cloth()
    x0 = sc.x0
    T = np.array([0.03, -0.04, 0.0])  # |T| = 5 cm
    xt = x0 + T
    osc = oracle.OracleScene(sc)
    prm = oracle.params()
    xn, st, tr = oracle.handle_step(osc, prm, x0, xt, trace_iters=64)
    step = 0.5 * prm.gamma * prm.d_max
    assert st["converged"] == 1
    assert st["pairs_evaluated"] == 0 and st["active_contacts"] == 0
    assert st["iterations"] == math.ceil(0.05 / step)
    assert st["searches"] == st["iterations"]
    assert np.array_equal(xn, xt)
    # each iterate lies on the segment toward the target: x^(l) - y = r (x^0 - y)
    for l in range(st["iterations"] + 1):
        d = tr["x"][l] - xt
        r = np.linalg.norm(d, axis=1) / np.linalg.norm(x0 - xt, axis=1)
        assert np.allclose(d, r[:, None] * (x0 - xt), atol=1e-15, rtol=0)
        if l < st["iterations"]:
            assert np.allclose(r, max(0.0, 1.0 - l * step / 0.05), atol=1e-12)


def test_p4_one_iteration_exact():
    sc = free_cloth()
    rng = np.random.default_rng(3)
    x0 = sc.x0
    xt = x0 + rng.uniform(-1, 1, size=x0.shape) * (0.4 * 4e-3 / np.sqrt(3.0))
    xn, st, _ = oracle.handle_step(oracle.OracleScene(sc), oracle.params(), x0, xt)
    assert st["iterations"] == 1 and st["converged"] == 1 and st["searches"] == 1
    assert np.array_equal(xn, xt)


@pytest.mark.parametrize("solver", [0, 1])
@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_p4b_non_finite_target_does_not_move(solver, bad):
    sc = free_cloth()
    rng = np.random.default_rng(4)
    x0 = sc.x0
    xt = x0 + rng.uniform(-1, 1, size=x0.shape) * (0.4 * 4e-3 / np.sqrt(3.0))
    k = 37
    xt[k] = [bad, 0.0, bad]
    prm = oracle.params(max_iters=5, solver=solver)
    xn, st, _ = oracle.handle_step(oracle.OracleScene(sc), prm, x0, xt)
    assert np.array_equal(xn[k], x0[k])
    others = np.arange(len(x0)) != k
    assert np.array_equal(xn[others], xt[others])
    assert st["converged"] == 0 and st["iterations"] == prm.max_iters + 1


def test_r2b_vertex_closer_than_the_floor_does_not_move():
    # R2b: a vertex 5e-11 m above a fixed triangle (below the 1e-10 floor)
    # keeps its position, although its target slides 1 mm along the plane
    from types import SimpleNamespace as NS
    x = np.array([[-0.1, -0.1, 0.0], [0.1, -0.1, 0.0], [0.0, 0.1, 0.0], [0.0, 0.0, 5e-11]])
    sc = NS(n_verts=4, inv_mass=np.array([0.0, 0.0, 0.0, 1.0]), radius=None, tris=np.array([[0, 1, 2]], np.int32),
            edges=np.zeros((0, 2), np.int32), len_edges=np.zeros((0, 2), np.int32), points=np.array([3], np.int32))
    xt = x.copy()
    xt[3, 0] += 1e-3
    xn, st, _ = oracle.handle_step(oracle.OracleScene(sc), oracle.params(max_iters=0), x, xt)
    assert np.array_equal(xn, x) and st["final_r_inf"] == 1.0
    # at 2e-10 (above the floor) it moves
    x[3, 2] = xt[3, 2] = 2e-10
    xn, st, _ = oracle.handle_step(oracle.OracleScene(sc), oracle.params(max_iters=0), x, xt)
    assert xn[3, 0] > 0.0


def colliding_cases():
    return [
        ("cloth_sphere", scenes.cloth_over_sphere(n=8, side=0.4, sphere_subdiv=1, sphere_r=0.12, noise=0.3, seed=5)),
        ("two_cloths", scenes.two_cloths(n=14, side=0.12, sep=0.003, omega=8.0, noise=0.3, seed=6)),
        ("hair_sand", scenes.hair_sand(n_strands=16, segs=6, n_points=40, grain_r=0.002, bowl_r=0.1, bowl_subdiv=2,
                                       seg_len=0.01, seed=7)),
    ]


@pytest.mark.parametrize("case", range(3))
def test_p5_safety_invariants(case):
    name, sc = colliding_cases()[case]
    osc = oracle.OracleScene(sc)
    prm = oracle.params_for(sc, max_iters=120)
    x, xt, v = scenes.initial(sc)
    assert oracle.count_intersections(osc, x) == 0
    for step in range(2):
        cap_p = 20000
        xn, st, tr = oracle.handle_step(osc, prm, x, xt, trace_iters=prm.max_iters + 2, trace_pairs=cap_p)
        L = st["iterations"]
        for l in range(L):
            xl, xl1 = tr["x"][l], tr["x"][l + 1]
            mv = np.linalg.norm(xl1 - xl, axis=1)
            Di = tr["Di"][l]
            assert np.all((mv < 0.5 * Di) | (mv == 0.0)), (name, step, l)
            Dl = tr["Dl"][l]
            assert tr["n_pairs"][l] <= cap_p
            held = set(tr["pair_keys"][l][:tr["n_pairs"][l]].tolist())
            fresh, _ = oracle.proximity(osc, xl, Dl, mode=0, x_tilde=xt)
            assert set(fresh.tolist()) <= held, (name, step, l)
            if l % 7 == 0:
                # CCD over every pair that could come within reach this iteration
                near, _ = oracle.proximity(osc, xl, 2.0 * Dl, mode=0, x_tilde=xt)
                for k in near.tolist():
                    kind, a, b = k >> 62, (k >> 31) & 0x7FFFFFFF, k & 0x7FFFFFFF
                    if kind == 0:
                        vs = [a, *sc.tris[b]]
                    elif kind == 1:
                        vs = [*sc.edges[a], *sc.edges[b]]
                    else:
                        vs = [a, b]
                    hit, _ = oracle.ccd(kind, xl[vs], xl1[vs])
                    assert not hit, (name, step, l, k)
        assert oracle.count_intersections(osc, xn) == 0
        if st["converged"]:
            assert st["final_r_inf"] < prm.eps
        assert L <= prm.max_iters + 1
        v = scenes.next_velocity(sc, xn, x)
        x, xt = xn, scenes.predict(sc, xn, v)


def test_jacobi_variant_is_safe():
    name, sc = colliding_cases()[1]
    osc = oracle.OracleScene(sc)
    x, xt, _ = scenes.initial(sc)
    for omega in (0.3, 0.6):
        prm = oracle.params_for(sc, max_iters=150, solver=1, jacobi_omega=omega)
        xn, st, _ = oracle.handle_step(osc, prm, x, xt)
        assert oracle.count_intersections(osc, xn) == 0
        assert st["iterations"] >= 1
