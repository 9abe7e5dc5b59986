"""Projected Jacobi backward step (Sec. 4.3.2) on the GPU against the oracle.

The per-vertex sums are segmented reductions in canonical key order, so the
FP64 path must follow the oracle step for step: same iteration counts, same
proximity sets, positions within 1e-9 relative (bitwise is expected).
"""
import numpy as np
import pytest

import oracle
from paper_2211_04045_gb300 import cch, scenes

from test_gpu_parity import REL, T, small_scenes

pytestmark = pytest.mark.gpu


def chain(cuda, sc, steps, **kw):
    gpu = cch.Scene(sc, cch.params_for(sc, **kw))
    osc = oracle.OracleScene(sc)
    oprm = oracle.params_for(sc, **kw)
    x, xt, _ = scenes.initial(sc)
    for s in range(steps):
        xo, so, _ = oracle.handle_step(osc, oprm, x, xt)
        out, sg = gpu.step(T(x, cuda), T(xt, cuda))
        xn = out.cpu().numpy()
        err = float(np.max(np.abs(xn - xo)))
        assert err <= REL * max(1.0, float(np.max(np.abs(xo)))), (s, err)
        assert sg["iterations"] == so["iterations"], (s, sg["iterations"], so["iterations"])
        assert sg["pairs_evaluated"] == so["pairs_evaluated"], s
        assert sg["active_contacts"] == so["active_contacts"], s
        assert sg["converged"] == so["converged"]
        assert oracle.count_intersections(osc, xn) == 0
        v = scenes.next_velocity(sc, xo, x)
        x, xt = xo, scenes.predict(sc, xo, v)
    gpu.close()


@pytest.mark.parametrize("name", list(small_scenes()))
def test_jacobi_chain_matches_oracle(cuda, name):
    chain(cuda, small_scenes()[name](), 2, max_iters=250, solver=1, jacobi_omega=0.5)


@pytest.mark.parametrize("name,omega,sweeps", [("two_cloths", 0.4, 3), ("tets", 0.7, 2), ("hair_sand", 0.5, 4)])
def test_jacobi_multi_sweep_matches_oracle(cuda, name, omega, sweeps):
    chain(cuda, small_scenes()[name](), 1, max_iters=200, solver=1, jacobi_omega=omega, gs_sweeps=sweeps)


@pytest.mark.parametrize("name", ["cloth_sphere", "two_cloths", "hair_sand"])
def test_jacobi_mixed_is_safe(cuda, name):
    sc = small_scenes()[name]()
    kw = dict(max_iters=250, solver=1, jacobi_omega=0.5)
    gpu = cch.Scene(sc, cch.params_for(sc, precision=1, accept_check=1, **kw))
    osc = oracle.OracleScene(sc)
    x, xt, _ = scenes.initial(sc)
    xo, so, _ = oracle.handle_step(osc, oracle.params_for(sc, **kw), x, xt)
    out, sg = gpu.step(T(x, cuda), T(xt, cuda))
    xm = out.cpu().numpy()
    travel = float(np.max(np.linalg.norm(xt - x, axis=1)))
    err = float(np.max(np.linalg.norm(xm - xo, axis=1)))
    print(f"{name}: mixed Jacobi vs FP64 oracle max |dx| = {err:.3e} m (travel {travel:.3e} m)")
    assert sg["intersections"] == 0 and sg["uncertain"] == 0
    assert oracle.count_intersections(osc, xm) == 0
    assert err <= 0.5 * travel + 1e-6
    gpu.close()


def test_jacobi_batch_equals_single(cuda):
    mk = small_scenes()
    scs = [mk["cloth_sphere"](), mk["two_cloths"](), mk["tets"]()]
    kw = dict(max_iters=200, solver=1, jacobi_omega=0.5)
    singles, inputs = [], []
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
        assert s1["iterations"] == s2["iterations"]
    b.close()
