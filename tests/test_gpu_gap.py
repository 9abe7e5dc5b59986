"""Gap-constraint variant (the comparison constraints of Sec. 4.1's gap
figure) on the GPU against the oracle: same iterations, positions within
1e-9 relative (bitwise expected), no intersection; mixed precision safe."""
import numpy as np
import pytest

import oracle
from paper_2211_04045_gb300 import cch, scenes

from test_gpu_parity import REL, T, small_scenes

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", list(small_scenes()))
def test_gap_chain_matches_oracle(cuda, name):
    sc = small_scenes()[name]()
    kw = dict(max_iters=250, constraint_form=1)
    gpu = cch.Scene(sc, cch.params_for(sc, **kw))
    osc = oracle.OracleScene(sc)
    oprm = oracle.params_for(sc, **kw)
    x, xt, _ = scenes.initial(sc)
    for s in range(2):
        xo, so, _ = oracle.handle_step(osc, oprm, x, xt)
        out, sg = gpu.step(T(x, cuda), T(xt, cuda))
        xn = out.cpu().numpy()
        err = float(np.max(np.abs(xn - xo)))
        assert err <= REL * max(1.0, float(np.max(np.abs(xo)))), (s, err)
        assert sg["iterations"] == so["iterations"] and sg["active_contacts"] == so["active_contacts"]
        assert oracle.count_intersections(osc, xn) == 0
        v = scenes.next_velocity(sc, xo, x)
        x, xt = xo, scenes.predict(sc, xo, v)
    gpu.close()


@pytest.mark.parametrize("name", ["two_cloths", "tets"])
def test_gap_mixed_is_safe(cuda, name):
    sc = small_scenes()[name]()
    gpu = cch.Scene(sc, cch.params_for(sc, max_iters=250, constraint_form=1, precision=1, accept_check=1))
    x, xt, _ = scenes.initial(sc)
    out, st = gpu.step(T(x, cuda), T(xt, cuda))
    assert st["intersections"] == 0 and st["uncertain"] == 0
    assert oracle.count_intersections(oracle.OracleScene(sc), out.cpu().numpy()) == 0
    gpu.close()
