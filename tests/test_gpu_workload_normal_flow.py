"""The normal-flow workload of Sec. 7.4 on the GPU against the oracle: the
same collision-handling kernels on closed tori whose targets self-intersect
(a shrinking tube and a closing hole).  Positions within 1e-9 relative
(bitwise expected), equal iterations and contacts, every state
intersection-free."""
import numpy as np
import pytest

import oracle
from paper_2211_04045_gb300 import cch, scenes

from test_gpu_parity import REL, T
from test_normal_flow_workload import flow_cases

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", list(flow_cases()))
def test_normal_flow_matches_oracle(cuda, name):
    sc = flow_cases()[name]()
    gpu = cch.Scene(sc, cch.params_for(sc))
    osc = oracle.OracleScene(sc)
    oprm = oracle.params_for(sc)
    x = sc.x0.copy()
    for step in range(3):
        y = scenes.predict(sc, x, None)
        xo, so, _ = oracle.handle_step(osc, oprm, x, y)
        out, sg = gpu.step(T(x, cuda), T(y, cuda))
        xn = out.cpu().numpy()
        err = float(np.max(np.abs(xn - xo)))
        assert err <= REL * max(1.0, float(np.max(np.abs(xo)))), (name, step, err)
        for k in ("iterations", "searches", "pairs_evaluated", "active_contacts", "converged"):
            assert sg[k] == so[k], (name, step, k, sg[k], so[k])
        assert oracle.count_intersections(osc, xn) == 0
        x = xo
    gpu.close()
