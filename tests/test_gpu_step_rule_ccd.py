"""CCD-based step size (the comparison scheme of Sec. 5.1) and the CCD
safety check with rounds, on the GPU against the oracle: positions within
1e-9 relative (bitwise expected: the CCD roots, clamps and steps are the
same operations on both sides), equal iterations and CCD hit counts."""
import numpy as np
import pytest

import oracle
from paper_2211_04045_gb300 import cch, scenes

from test_gpu_parity import REL, T, small_scenes

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", list(small_scenes()))
def test_ccd_rule_matches_oracle(cuda, name):
    sc = small_scenes()[name]()
    kw = dict(max_iters=120, step_rule=1)
    gpu = cch.Scene(sc, cch.params_for(sc, **kw))
    osc = oracle.OracleScene(sc)
    x, xt, _ = scenes.initial(sc)
    xo, so, _ = oracle.handle_step(osc, oracle.params_for(sc, **kw), x, xt)
    out, sg = gpu.step(T(x, cuda), T(xt, cuda))
    xn = out.cpu().numpy()
    err = float(np.max(np.abs(xn - xo)))
    assert err <= REL * max(1.0, float(np.max(np.abs(xo)))), (name, err)
    for k in ("iterations", "searches", "pairs_evaluated", "active_contacts", "ccd_clamps", "converged"):
        assert sg[k] == so[k], (name, k, sg[k], so[k])
    assert oracle.count_intersections(osc, xn) == 0
    gpu.close()


@pytest.mark.parametrize("rounds", [0, 1])
@pytest.mark.parametrize("name", ["cloth_sphere", "two_cloths"])
def test_few_rounds_match_oracle(cuda, name, rounds):
    # with 0 or 1 clamp rounds a remaining hit keeps the scene in place for
    # the iteration (the freeze path), on both sides
    sc = small_scenes()[name]()
    kw = dict(max_iters=80, step_rule=1, ccd_rounds=rounds)
    gpu = cch.Scene(sc, cch.params_for(sc, **kw))
    osc = oracle.OracleScene(sc)
    x, xt, _ = scenes.initial(sc)
    xo, so, _ = oracle.handle_step(osc, oracle.params_for(sc, **kw), x, xt)
    out, sg = gpu.step(T(x, cuda), T(xt, cuda))
    xn = out.cpu().numpy()
    assert float(np.max(np.abs(xn - xo))) <= REL * max(1.0, float(np.max(np.abs(xo))))
    assert sg["iterations"] == so["iterations"] and sg["ccd_clamps"] == so["ccd_clamps"]
    assert oracle.count_intersections(osc, xn) == 0
    gpu.close()


@pytest.mark.parametrize("name", ["cloth_sphere", "two_cloths"])
def test_safety_check_changes_nothing(cuda, name):
    sc = small_scenes()[name]()
    x, xt, _ = scenes.initial(sc)
    outs = []
    for check in (0, 1):
        gpu = cch.Scene(sc, cch.params_for(sc, max_iters=120, ccd_check=check))
        out, st = gpu.step(T(x, cuda), T(xt, cuda))
        outs.append((out.cpu().numpy(), st))
        gpu.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[1][1]["ccd_clamps"] == 0 and outs[0][1]["iterations"] == outs[1][1]["iterations"]


def test_ccd_rule_batch_equals_single(cuda):
    mk = small_scenes()
    scs = [mk["cloth_sphere"](), mk["two_cloths"](), mk["tets"]()]
    kw = dict(max_iters=100, step_rule=1)
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
        assert s1["iterations"] == s2["iterations"] and s1["ccd_clamps"] == s2["ccd_clamps"]
    b.close()
