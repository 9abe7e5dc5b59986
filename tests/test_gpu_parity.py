"""CUDA path against the CPU oracle, element by element (FP64 mode).

Candidate sets and proximity sets must match bit-exactly (keys and
distances); positions after a step must match to 1e-9 relative (bitwise is
expected, since both sides evaluate the same arithmetic without contraction).
"""
import numpy as np
import pytest

import oracle
from paper_2211_04045_gb300 import cch, scenes

pytestmark = pytest.mark.gpu

REL = 1e-9


def small_scenes():
    return {
        "cloth_sphere": lambda: scenes.cloth_over_sphere(n=10, side=0.5, sphere_subdiv=1, sphere_r=0.15, noise=0.3,
                                                         seed=1),
        "two_cloths": lambda: scenes.two_cloths(n=24, side=0.25, sep=0.004, omega=6.0, noise=0.3, seed=2),
        "tets": lambda: scenes.tet_bodies(n_bodies=8, n=4, side=0.08, box=0.32, v_sigma=2.0, w_sigma=4.0, seed=3),
        "knot": lambda: scenes.tube_knot(around=12, rings=41, r=0.004, helix_r=0.0055, pitch=0.03, ring_dz=0.002),
        "hair_sand": lambda: scenes.hair_sand(n_strands=36, segs=8, n_points=120, grain_r=0.002, bowl_r=0.12,
                                              bowl_subdiv=2, seg_len=0.01, seed=4),
    }


def T(a, dev):
    import torch
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)


# statistics of the Gauss-Seidel colouring and of the forward step that must
# equal the oracle's
GS_STATS = ("contact_colours", "edge_colours", "contact_vertices", "frozen_vertices", "max_vertex_contacts",
            "max_vertex_edges", "degenerate", "pair_vertices")


def same_stats(sg, so, where):
    for k in GS_STATS:
        assert sg[k] == so[k], (where, k, sg[k], so[k])


def jitter(x, scale, seed):
    rng = np.random.default_rng(seed)
    return x + rng.normal(0.0, scale, size=x.shape)


@pytest.mark.parametrize("name", list(small_scenes()))
def test_candidate_and_proximity_sets_bit_exact(cuda, name):
    sc = small_scenes()[name]()
    x0, xt, _ = scenes.initial(sc)
    prm = cch.params_for(sc)
    gpu = cch.Scene(sc, prm)
    osc = oracle.OracleScene(sc)
    states = [x0, jitter(x0, 0.002, 10), jitter(xt, 0.004, 11)]
    for k, x in enumerate(states):
        for D in (prm.d_max, 3.0 * prm.d_max):
            gk, _ = gpu.query_pairs(T(x, cuda), T(xt, cuda), D, candidates=True)
            ok = oracle.candidates(osc, x, D, mode=0, x_tilde=xt)
            assert np.array_equal(gk, ok), (name, k, D, len(gk), len(ok))
            gk, gd = gpu.query_pairs(T(x, cuda), T(xt, cuda), D, candidates=False)
            ok, od = oracle.proximity(osc, x, D, mode=0, x_tilde=xt)
            assert np.array_equal(gk, ok), (name, k, D, len(gk), len(ok))
            assert np.array_equal(gd, od), (name, k, D, float(np.max(np.abs(gd - od))) if len(gd) else 0)
    gpu.close()


@pytest.mark.parametrize("colouring", [1, 0])
@pytest.mark.parametrize("name", list(small_scenes()))
def test_step_chain_matches_oracle(cuda, name, colouring):
    sc = small_scenes()[name]()
    steps = 3
    prm_kw = dict(max_iters=300, colouring=colouring)
    gpu = cch.Scene(sc, cch.params_for(sc, **prm_kw))
    osc = oracle.OracleScene(sc)
    oprm = oracle.params_for(sc, **prm_kw)
    x, xt, v = scenes.initial(sc)
    xg, xtg, vg = x.copy(), xt.copy(), v.copy()
    for s in range(steps):
        xo, so, _ = oracle.handle_step(osc, oprm, x, xt)
        out, sg = gpu.step(T(xg, cuda), T(xtg, cuda))
        xn = out.cpu().numpy()
        scale = max(1.0, float(np.max(np.abs(xo))))
        err = float(np.max(np.abs(xn - xo)))
        assert err <= REL * scale, (name, s, err)
        assert sg["iterations"] == so["iterations"], (name, s, sg["iterations"], so["iterations"])
        assert sg["searches"] == so["searches"], (name, s)
        assert sg["pairs_evaluated"] == so["pairs_evaluated"], (name, s)
        assert sg["active_contacts"] == so["active_contacts"], (name, s)
        assert sg["converged"] == so["converged"]
        same_stats(sg, so, (name, s))
        v = scenes.next_velocity(sc, xo, x)
        x, xt = xo, scenes.predict(sc, xo, v)
        vg = scenes.next_velocity(sc, xn, xg)
        xg, xtg = xn, scenes.predict(sc, xn, vg)
    gpu.close()


def test_tiny_move_is_one_iteration_and_exact(cuda):
    # P4: every move below 0.45 D^max and no pair within D^max: one iteration, x^{t+1} == x~ bitwise
    sc = scenes.two_cloths(n=16, side=0.3, sep=0.05, omega=0.0, noise=0.0)
    x0 = sc.x0
    rng = np.random.default_rng(5)
    xt = x0 + rng.uniform(-1.0, 1.0, size=x0.shape) * (0.4 * 4e-3 / np.sqrt(3.0))
    gpu = cch.Scene(sc, cch.params_for(sc))
    out, st = gpu.step(T(x0, cuda), T(xt, cuda))
    assert st["iterations"] == 1 and st["converged"] == 1
    assert np.array_equal(out.cpu().numpy(), xt)
    gpu.close()


def test_batch_equals_single(cuda):
    mk = small_scenes()
    scs = [mk["cloth_sphere"](), mk["two_cloths"](), mk["tets"]()]
    kw = dict(max_iters=200)
    singles = []
    inputs = []
    for sc in scs:
        x, xt, _ = scenes.initial(sc)
        g = cch.Scene(sc, cch.params_for(sc, **kw))
        o, st = g.step(T(x, cuda), T(xt, cuda))
        singles.append((o.cpu().numpy(), st))
        inputs.append((x, xt))
        g.close()
    b = cch.Scene(scs, cch.params_for(scs[0], **kw))
    outs, sts = b.batch_step([T(a, cuda) for a, _ in inputs], [T(c, cuda) for _, c in inputs])
    for (o1, s1), o2, s2 in zip(singles, outs, sts):
        assert np.array_equal(o1, o2.cpu().numpy())
        assert s1["iterations"] == s2["iterations"] and s1["pairs_evaluated"] == s2["pairs_evaluated"]
    b.close()
