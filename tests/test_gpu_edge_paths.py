"""Paths of the CUDA library that the workload-sized tests do not reach,
each against the oracle: pair buffers that overflow, grow and replay the
step; the branch for more than 32 items per thread of the colouring and of
both sweeps (forced with a one-block cooperative grid); Gauss-Seidel with
several sweeps per backward step (Sec. 4.3.1); and a bounded device wait that
runs out, after which the same scene completes a normal step.  Every
Gauss-Seidel case runs with both colourings (level and greedy).
"""
import numpy as np
import pytest

import oracle
from paper_2211_04045_gb300 import cch, scenes

from test_gpu_parity import REL, T, same_stats, small_scenes

pytestmark = pytest.mark.gpu


def one_step(cuda, sc, x, xt, gpu, **kw):
    xo, so, _ = oracle.handle_step(oracle.OracleScene(sc), oracle.params_for(sc, **kw), x, xt)
    out, sg = gpu.step(T(x, cuda), T(xt, cuda))
    xn = out.cpu().numpy()
    err = float(np.max(np.abs(xn - xo)))
    assert err <= REL * max(1.0, float(np.max(np.abs(xo)))), err
    for k in ("iterations", "searches", "pairs_evaluated", "active_contacts", "converged"):
        assert sg[k] == so[k], (k, sg[k], so[k])
    return xn, sg, so


def test_pair_buffers_grow_and_the_step_replays(cuda):
    # buffers of 64 pairs: every search overflows them, the library doubles
    # them and runs the step again from its inputs
    sc = scenes.two_cloths(n=24, side=0.25, sep=0.004, omega=6.0, noise=0.3, seed=2)
    kw = dict(max_iters=300)
    small = cch.Scene(sc, cch.params_for(sc, pair_capacity=64, **kw))
    ref = cch.Scene(sc, cch.params_for(sc, **kw))
    x, xt, _ = scenes.initial(sc)
    for s in range(2):
        xn, sg, so = one_step(cuda, sc, x, xt, small, **kw)
        assert so["max_pairs"] > 64
        same_stats(sg, so, s)
        o2, _ = ref.step(T(x, cuda), T(xt, cuda))
        assert np.array_equal(xn, o2.cpu().numpy())
        v = scenes.next_velocity(sc, xn, x)
        x, xt = xn, scenes.predict(sc, xn, v)
    small.close()
    ref.close()


@pytest.mark.parametrize("colouring", [1, 0])
def test_more_than_32_items_per_thread(cuda, colouring):
    # two 48 x 48 layers 0.7 mm apart: 13,442 edge-length constraints and
    # more than 8,192 contacts, against a grid of one block of 256 threads
    # (32 x 256 = 8,192 items per list)
    sc = scenes.two_cloths(n=48, side=0.4, sep=0.0007, omega=6.0, noise=0.3, seed=3)
    assert len(sc.len_edges) > 8192
    kw = dict(max_iters=24, colouring=colouring)
    one = cch.Scene(sc, cch.params_for(sc, sweep_blocks=1, **kw))
    full = cch.Scene(sc, cch.params_for(sc, **kw))
    x, xt, _ = scenes.initial(sc)
    xn, sg, so = one_step(cuda, sc, x, xt, one, **kw)
    same_stats(sg, so, "one block")
    _, _, tr = oracle.handle_step(oracle.OracleScene(sc), oracle.params_for(sc, **kw), x, xt, trace_iters=32)
    assert int(np.max(tr["n_contacts"])) > 8192
    o2, s2 = full.step(T(x, cuda), T(xt, cuda))
    assert np.array_equal(xn, o2.cpu().numpy()) and s2["iterations"] == sg["iterations"]
    one.close()
    full.close()


def test_full_quad_lists_of_the_level_sweep(cuda):
    # the FP64 level sweep gives each quad of lanes up to 4 x 32 items; with a
    # one-block grid (64 quads) a scene of 4,096-8,192 items fills them to
    # 16-32 items per lane, against the same step on the full grid
    sc = scenes.two_cloths(n=32, side=0.3, sep=0.0012, omega=6.0, noise=0.3, seed=4)
    kw = dict(max_iters=40)
    _, _, tr = oracle.handle_step(oracle.OracleScene(sc), oracle.params_for(sc, **kw), *scenes.initial(sc)[:2],
                                  trace_iters=48)
    items = np.asarray(tr["n_contacts"]) + len(sc.len_edges)
    assert 4096 < items.min() and items.max() <= 8192, (items.min(), items.max())
    one = cch.Scene(sc, cch.params_for(sc, sweep_blocks=1, **kw))
    full = cch.Scene(sc, cch.params_for(sc, **kw))
    x, xt, _ = scenes.initial(sc)
    xn, sg, so = one_step(cuda, sc, x, xt, one, **kw)
    same_stats(sg, so, "one block")
    o2, s2 = full.step(T(x, cuda), T(xt, cuda))
    assert np.array_equal(xn, o2.cpu().numpy()) and s2["iterations"] == sg["iterations"]
    one.close()
    full.close()


@pytest.mark.parametrize("colouring", [1, 0])
@pytest.mark.parametrize("sweeps", [2, 3])
@pytest.mark.parametrize("name", ["cloth_sphere", "two_cloths", "tets"])
def test_gauss_seidel_several_sweeps(cuda, name, sweeps, colouring):
    sc = small_scenes()[name]()
    kw = dict(max_iters=300, gs_sweeps=sweeps, colouring=colouring)
    gpu = cch.Scene(sc, cch.params_for(sc, **kw))
    x, xt, _ = scenes.initial(sc)
    for s in range(2):
        xn, sg, so = one_step(cuda, sc, x, xt, gpu, **kw)
        same_stats(sg, so, (name, sweeps, s))
        v = scenes.next_velocity(sc, xn, x)
        x, xt = xn, scenes.predict(sc, xn, v)
    gpu.close()


@pytest.mark.parametrize("colouring", [1, 0])
def test_bounded_wait_runs_out_and_the_scene_recovers(cuda, colouring):
    # layers 0.7 mm apart: the first iteration already has contacts that
    # share vertices, so the sweep (level colouring) or the colouring pass
    # (greedy) waits on its counters
    sc = scenes.two_cloths(n=24, side=0.25, sep=0.0007, omega=6.0, noise=0.3, seed=5)
    kw = dict(max_iters=40, colouring=colouring)
    gpu = cch.Scene(sc, cch.params_for(sc, **kw))
    x, xt, _ = scenes.initial(sc)
    gpu.set_max_polls(1)
    with pytest.raises(cch.CchError) as e:
        gpu.step(T(x, cuda), T(xt, cuda))
    assert e.value.code == 6  # CCH_E_TIMEOUT
    gpu.set_max_polls(0)
    one_step(cuda, sc, x, xt, gpu, **kw)
    gpu.close()
