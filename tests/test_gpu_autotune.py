"""Autotuner of the launch configuration: it picks
from the stated candidate sets, every probe gives the same result, and steps
after tuning equal steps before it bitwise (the configuration never changes
results)."""
import numpy as np
import pytest

from paper_2211_04045_gb300 import cch, scenes

pytestmark = pytest.mark.gpu


def T(a, dev):
    import torch
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)


@pytest.mark.parametrize("solver", [0, 1])
def test_autotune_choice_and_identical_results(cuda, solver):
    sc = scenes.two_cloths(n=32, side=0.3, sep=0.004, omega=6.0, noise=0.3, seed=7)
    x, xt, _ = scenes.initial(sc)
    g = cch.Scene(sc, cch.params_for(sc, max_iters=120, solver=solver))
    before, st0 = g.step(T(x, cuda), T(xt, cuda))
    r = g.autotune(T(x, cuda), T(xt, cuda), probe_iters=24)
    assert r["consistent"] == 1
    assert r["iters_per_launch"] in (4, 8, 16, 32, 64)
    assert r["query_block"] in (64, 128, 256)
    assert r["bvh_refit_only"] in (0, 1)
    assert r["packet_traversal"] in (0, 1)
    assert r["trials"] >= 8
    assert 0 < r["best_ms"] <= r["default_ms"]
    after, st1 = g.step(T(x, cuda), T(xt, cuda))
    assert np.array_equal(before.cpu().numpy(), after.cpu().numpy())
    assert st0["iterations"] == st1["iterations"] and st0["pairs_evaluated"] == st1["pairs_evaluated"]
    g.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("which", ["cloth_sphere", "two_cloths"])
def test_bvh_rebuild_equals_refit(cuda, precision, which):
    # rebuilding the BVH at every search changes the tree, not the pairs and
    # not their distances (in mixed precision the FP32 bound is the distance,
    # so it must not depend on which primitive is the query)
    if which == "cloth_sphere":
        sc = scenes.cloth_over_sphere(n=12, side=0.5, sphere_subdiv=2, sphere_r=0.15, noise=0.3, seed=8)
    else:
        sc = scenes.two_cloths(n=24, side=0.25, sep=0.004, omega=6.0, noise=0.3, seed=2)
    x, xt, _ = scenes.initial(sc)
    outs = []
    for refit in (1, 0):
        g = cch.Scene(sc, cch.params_for(sc, max_iters=150, bvh_refit_only=refit, precision=precision))
        o, st = g.step(T(x, cuda), T(xt, cuda))
        outs.append((o.cpu().numpy(), st["iterations"], st["pairs_evaluated"]))
        g.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1:] == outs[1][1:]
