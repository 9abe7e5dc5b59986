"""Convergence of the oracle in the paper's regime (Table 2's text: the loop
typically converges in less than 64 steps; termination on ||r||_inf < eps,
Algorithm 1).  Two spinning cloth layers at dt = 1/100 (the paper's step for
most examples): with or without velocity noise, every step of a chain of four
converges within 64 iterations, with no vertex held by the D_i floor, and the
result is intersection-free.  Without noise and contacts the count is the
travel bound: ceil(largest move / (0.45 D^max)) plus the final iteration.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2211_04045_gb300 import scenes


@pytest.mark.parametrize("noise,seed", [(0.0, 0), (0.3, 0), (0.3, 1)])
def test_spinning_cloths_converge_within_64_iterations(noise, seed):
    sc = scenes.two_cloths(n=32, side=0.25, sep=0.01, omega=6.0, noise=noise, seed=seed, dt=1.0 / 100)
    osc = oracle.OracleScene(sc)
    prm = oracle.params_for(sc)
    x, xt, v = scenes.initial(sc)
    for s in range(4):
        xn, st, _ = oracle.handle_step(osc, prm, x, xt)
        assert st["converged"] == 1 and st["iterations"] < 64, (noise, seed, s, st["iterations"])
        assert st["final_r_inf"] < prm.eps and st["frozen_vertices"] == 0
        assert oracle.count_intersections(osc, xn) == 0
        if noise == 0.0 and st["active_contacts"] == 0:
            far = float(np.max(np.linalg.norm(xt - x, axis=1)))
            assert st["iterations"] <= math.ceil(far / (0.45 * prm.d_max)) + 1
        v = scenes.next_velocity(sc, xn, x)
        x, xt = xn, scenes.predict(sc, xn, v)
