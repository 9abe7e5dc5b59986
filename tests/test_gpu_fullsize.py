"""Full-size workload (two 256 x 256 cloths, 131,072 vertices) on the GPU.

The candidate set and the proximity set at the generator's states are
compared with the oracle in full (the oracle's sorted-axis window search takes
seconds at this size).  A step capped at six iterations, from a contact-rich
state (the layers 1.5 mm apart, so that every vertex has pairs in P and
contacts form within the first iterations), is compared with the oracle
element by element: positions, iterations, searches, |P|, contacts and the
colouring's statistics (the oracle takes about ten seconds per iteration at
this size).  For whole steps, where the oracle would take hours, the test
checks properties that hold at any size: a repeated call is bitwise
identical, and the statistics are consistent.
"""
import numpy as np
import pytest

import oracle
from paper_2211_04045_gb300 import cch, scenes

pytestmark = pytest.mark.gpu


def T(a, dev):
    import torch
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)


@pytest.fixture(scope="module")
def c2():
    return scenes.two_cloths(n=256, side=2.0, sep=0.01, omega=6.0, noise=0.3, seed=0)


def test_fullsize_pair_sets_bit_exact(cuda, c2):
    x0, xt, _ = scenes.initial(c2)
    gpu = cch.Scene(c2, cch.params_for(c2))
    osc = oracle.OracleScene(c2)
    D = 4e-3
    for x in (x0, xt):
        gk, _ = gpu.query_pairs(T(x, cuda), T(xt, cuda), D, candidates=True)
        ok = oracle.candidates(osc, x, D, mode=1, x_tilde=xt)
        assert len(ok) > 10000
        assert np.array_equal(gk, ok)
        gk, gd = gpu.query_pairs(T(x, cuda), T(xt, cuda), D, candidates=False)
        ok, od = oracle.proximity(osc, x, D, mode=1, x_tilde=xt)
        assert np.array_equal(gk, ok) and np.array_equal(gd, od)
    gpu.close()


@pytest.mark.parametrize("colouring", [1, 0])
def test_fullsize_capped_step_matches_oracle(cuda, colouring):
    from test_gpu_parity import REL, same_stats
    sc = scenes.two_cloths(n=256, side=2.0, sep=0.0015, omega=6.0, noise=0.3, seed=0)
    x, xt, _ = scenes.initial(sc)
    kw = dict(max_iters=5, colouring=colouring)
    xo, so, _ = oracle.handle_step(oracle.OracleScene(sc), oracle.params_for(sc, **kw), x, xt)
    gpu = cch.Scene(sc, cch.params_for(sc, **kw))
    out, sg = gpu.step(T(x, cuda), T(xt, cuda))
    xn = out.cpu().numpy()
    err = float(np.max(np.abs(xn - xo)))
    assert err <= REL * max(1.0, float(np.max(np.abs(xo)))), err
    for k in ("iterations", "searches", "pairs_evaluated", "max_pairs", "active_contacts", "converged"):
        assert sg[k] == so[k], (k, sg[k], so[k])
    same_stats(sg, so, "full size")
    assert so["iterations"] == 6 and so["pairs_evaluated"] > 10**7 and so["active_contacts"] > 1000
    gpu.close()


def test_fullsize_step_is_deterministic(cuda, c2):
    x0, xt, _ = scenes.initial(c2)
    gpu = cch.Scene(c2, cch.params_for(c2, max_iters=96))
    a, sa = gpu.step(T(x0, cuda), T(xt, cuda))
    b, sb = gpu.step(T(x0, cuda), T(xt, cuda))
    import torch
    assert torch.equal(a, b)
    assert sa["iterations"] == sb["iterations"] == 97
    assert sa["pairs_evaluated"] == sb["pairs_evaluated"] and sa["searches"] == sb["searches"]
    assert sa["searches"] >= 1 and sa["max_pairs"] > 0
    # every vertex moved at most its share of the 0.45 D^max per iteration bound
    moved = torch.linalg.norm(a - T(x0, cuda), dim=1).max().item()
    assert moved <= 0.45 * 4e-3 * sa["iterations"] * (1 + 1e-12)
    gpu.close()


def test_hair_sand_fullsize_sampled_pairs(cuda):
    # Full-size hair and sand (10,000 strands x 32 segments, 100,000 grains of
    # radius 2 mm, a fixed bowl), the movable vertices jittered by 1.5 mm so
    # that strands and grains come within D^max = 0.8 mm of each other.  The
    # oracle's whole-scene search takes hours here, so sampled queries are
    # checked one by one (pair_sampling.check_sampled_pairs): for 1,000
    # collision vertices, 1,000 edges and 1,000 grains the GPU's pairs in P
    # are recomputed with the oracle's distance routines.
    from pair_sampling import check_sampled_pairs, jittered
    sc = scenes.hair_sand()
    x0, xt, _ = scenes.initial(sc)
    x = jittered(sc, x0, 0.0015, 7)
    D = float(cch.params_for(sc).d_max)
    gpu = cch.Scene(sc, cch.params_for(sc))
    gk, gd = gpu.query_pairs(T(x, cuda), T(xt, cuda), D, candidates=False)
    gpu.close()
    checked = check_sampled_pairs(sc, x, xt, D, dict(zip(gk.tolist(), gd.tolist())), 1000, seed=8)
    assert checked > 1000
