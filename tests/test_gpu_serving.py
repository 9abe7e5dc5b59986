"""Serving: resident scenes, requests arriving while
others run, continuous batching at launch boundaries.  Each result must equal
the result of the same request run alone, bitwise, in FP64 and in mixed
precision, with either backward step (every path is deterministic)."""
import time

import numpy as np
import pytest

from paper_2211_04045_gb300 import cch, scenes

pytestmark = pytest.mark.gpu


def T(a, dev):
    import torch
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)


@pytest.mark.parametrize("precision,solver", [(0, 0), (1, 0), (0, 1)])
def test_served_results_equal_single_results(cuda, precision, solver):
    import torch
    mk = [lambda: scenes.cloth_over_sphere(n=10, side=0.5, sphere_subdiv=1, sphere_r=0.15, noise=0.3, seed=1),
          lambda: scenes.two_cloths(n=24, side=0.25, sep=0.004, omega=6.0, noise=0.3, seed=2),
          lambda: scenes.tet_bodies(n_bodies=8, n=4, side=0.08, box=0.32, seed=3)]
    scs = [f() for f in mk]
    kw = dict(max_iters=150, iters_per_launch=4, precision=precision, solver=solver)
    # requests: two successive steps of each scene, plus repeats
    reqs = []
    for k, sc in enumerate(scs):
        x, xt, v = scenes.initial(sc)
        reqs.append((k, x, xt))
        x2 = xt + 0.001
        reqs.append((k, x, scenes.predict(sc, x, v * 0.5)))
    alone = []
    for k, x, xt in reqs:
        g = cch.Scene(scs[k], cch.params_for(scs[k], **kw))
        o, st = g.step(T(x, cuda), T(xt, cuda))
        alone.append((o.cpu().numpy(), st["iterations"]))
        g.close()
    sv = cch.Server(8 << 30, cch.params_for(scs[0], **kw), max_active=2)
    ids = [sv.add_scene(sc) for sc in scs]
    outs, tickets = [], []
    for i, (k, x, xt) in enumerate(reqs):
        o = torch.empty((scs[k].n_verts, 3), dtype=torch.float64, device=cuda)
        outs.append(o)
        tickets.append(sv.submit(ids[k], T(x, cuda), T(xt, cuda), o))
        time.sleep(0.002 * (i % 3))  # arrivals while earlier requests run
    lat = []
    for i, tk in enumerate(tickets):
        st, ms = sv.wait(tk)
        lat.append(ms)
        assert st["iterations"] == alone[i][1], i
        assert np.array_equal(outs[i].cpu().numpy(), alone[i][0]), i
    assert all(m > 0 for m in lat)
    sv.close()


def test_scenes_keep_their_own_parameters(cuda):
    # a tube pair (delta = 0.5 mm, D in [1, 2] mm) next to a cloth scene with
    # Table 2's defaults: served and batched with per-scene parameters, each
    # result equals the scene stepped alone with its own parameters
    import torch
    scs = [scenes.tube_knot(around=16, rings=65, r=0.004, helix_r=0.0055, pitch=0.03, ring_dz=0.002),
           scenes.two_cloths(n=24, side=0.25, sep=0.004, omega=6.0, noise=0.3, seed=2)]
    assert dict(scs[0].params)["delta"] != cch.params_for(scs[1]).delta
    kw = dict(max_iters=150, iters_per_launch=4)
    rng = np.random.default_rng(5)
    reqs = []
    for k, sc in enumerate(scs):
        x, xt, _ = scenes.initial(sc)
        reqs.append((k, x, x + rng.normal(0.0, 3e-4, x.shape) * (sc.inv_mass > 0)[:, None]))
    alone = []
    for k, x, xt in reqs:
        g = cch.Scene(scs[k], cch.params_for(scs[k], **kw))
        o, st = g.step(T(x, cuda), T(xt, cuda))
        alone.append((o.cpu().numpy(), st["iterations"], st["pairs_evaluated"]))
        g.close()
    sv = cch.Server(8 << 30, cch.params_for(scs[1], **kw), max_active=2)
    ids = [sv.add_scene(sc, cch.params_for(sc, **kw)) for sc in scs]
    outs = [torch.empty((scs[k].n_verts, 3), dtype=torch.float64, device=cuda) for k, _, _ in reqs]
    tickets = [sv.submit(ids[k], T(x, cuda), T(xt, cuda), outs[i]) for i, (k, x, xt) in enumerate(reqs)]
    for i, tk in enumerate(tickets):
        st, _ = sv.wait(tk)
        assert st["iterations"] == alone[i][1] and st["pairs_evaluated"] == alone[i][2], i
        assert np.array_equal(outs[i].cpu().numpy(), alone[i][0]), i
    sv.close()
    b = cch.Scene(scs, cch.params_for(scs[1], **kw), scene_params=[cch.params_for(sc, **kw) for sc in scs])
    outs, sts = b.batch_step([T(x, cuda) for _, x, _ in reqs], [T(xt, cuda) for _, _, xt in reqs])
    for i in range(len(reqs)):
        assert sts[i]["iterations"] == alone[i][1], i
        assert np.array_equal(outs[i].cpu().numpy(), alone[i][0]), i
    b.close()
