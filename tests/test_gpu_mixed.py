"""Mixed precision (FP32 distances, contacts and projection; FP64 forward
step, CCD and acceptance): safe, and close to the FP64 oracle.

The pair distances become FP32 lower bounds (d32 minus its rounding bound),
so every D_i stays below the true distance and the forward step keeps its
guarantee; the acceptance test and the oracle's exact test must both find
no intersection.  The position error against the FP64 oracle is reported
and bounded loosely: y only guides the forward step, so rounding differences
change the path, not its safety.
"""
import numpy as np
import pytest

import oracle
from paper_2211_04045_gb300 import cch, scenes

pytestmark = pytest.mark.gpu


def T(a, dev):
    import torch
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)


CASES = {
    "cloth_sphere": lambda: scenes.cloth_over_sphere(n=10, side=0.5, sphere_subdiv=1, sphere_r=0.15, noise=0.3,
                                                     seed=1),
    "two_cloths": lambda: scenes.two_cloths(n=24, side=0.25, sep=0.004, omega=6.0, noise=0.3, seed=2),
    "tets": lambda: scenes.tet_bodies(n_bodies=8, n=4, side=0.08, box=0.32, seed=3),
    "hair_sand": lambda: scenes.hair_sand(n_strands=36, segs=8, n_points=120, grain_r=0.002, bowl_r=0.12,
                                          bowl_subdiv=2, seg_len=0.01, seed=4),
}


@pytest.mark.parametrize("name", list(CASES))
def test_mixed_is_safe_and_close(cuda, name):
    sc = CASES[name]()
    kw = dict(max_iters=300)
    gpu = cch.Scene(sc, cch.params_for(sc, precision=1, accept_check=1, **kw))
    osc = oracle.OracleScene(sc)
    x, xt, _ = scenes.initial(sc)
    xo, so, _ = oracle.handle_step(osc, oracle.params_for(sc, **kw), x, xt)
    out, sg = gpu.step(T(x, cuda), T(xt, cuda))
    xm = out.cpu().numpy()
    err = float(np.max(np.linalg.norm(xm - xo, axis=1)))
    travel = float(np.max(np.linalg.norm(xt - x, axis=1)))
    print(f"{name}: mixed vs FP64 oracle max |dx| = {err:.3e} m (largest target move {travel:.3e} m), "
          f"iterations {sg['iterations']} vs {so['iterations']}")
    assert sg["intersections"] == 0 and sg["uncertain"] == 0
    assert oracle.count_intersections(osc, xm) == 0
    assert err <= 0.5 * travel + 1e-6
    gpu.close()
