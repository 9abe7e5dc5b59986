"""The rotating-sphere workload of Sec. 6.3 (friction by the velocity filter
on the target) on the GPU against the oracle: the filter runs on the host
in the input generator, the collision-handling step on both sides.
Positions within 1e-9 relative (bitwise expected), equal iterations and
contacts, every state intersection-free."""
import numpy as np
import pytest

import oracle
from paper_2211_04045_gb300 import cch, scenes

from test_gpu_parity import REL, T

pytestmark = pytest.mark.gpu


def test_rotating_sphere_with_friction_matches_oracle(cuda):
    sc = scenes.cloth_on_rotating_sphere(n=16, side=0.5, sphere_subdiv=2, sphere_r=0.15, omega=2.0, mu=0.5)
    gpu = cch.Scene(sc, cch.params_for(sc))
    osc = oracle.OracleScene(sc)
    oprm = oracle.params_for(sc)
    x, xt, v = scenes.initial(sc)
    for step in range(4):
        xo, so, _ = oracle.handle_step(osc, oprm, x, xt)
        out, sg = gpu.step(T(x, cuda), T(xt, cuda))
        xn = out.cpu().numpy()
        err = float(np.max(np.abs(xn - xo)))
        assert err <= REL * max(1.0, float(np.max(np.abs(xo)))), (step, err)
        for k in ("iterations", "searches", "pairs_evaluated", "active_contacts", "converged"):
            assert sg[k] == so[k], (step, k, sg[k], so[k])
        assert oracle.count_intersections(osc, xn) == 0
        v = scenes.next_velocity(sc, xo, x)
        x, xt = xo, scenes.predict(sc, xo, v)
    gpu.close()
