"""Segment CCD safety check (the CCD of Sec. 5.1's comparison scheme, used as
a check) and the acceptance test of x^{t+1} on the GPU, against the oracle."""
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
    "hair_sand": lambda: scenes.hair_sand(n_strands=36, segs=8, n_points=120, grain_r=0.002, bowl_r=0.12,
                                          bowl_subdiv=2, seg_len=0.01, seed=4),
}


@pytest.mark.parametrize("name", list(CASES))
def test_ccd_mode_and_acceptance_match_oracle(cuda, name):
    sc = CASES[name]()
    kw = dict(max_iters=200, ccd_check=1)
    gpu = cch.Scene(sc, cch.params_for(sc, accept_check=1, **kw))
    osc = oracle.OracleScene(sc)
    oprm = oracle.params_for(sc, **kw)
    x, xt, _ = scenes.initial(sc)
    for step in range(2):
        xo, so, _ = oracle.handle_step(osc, oprm, x, xt)
        out, sg = gpu.step(T(x, cuda), T(xt, cuda))
        xn = out.cpu().numpy()
        assert np.max(np.abs(xn - xo)) <= 1e-9 * max(1.0, np.max(np.abs(xo)))
        assert sg["ccd_clamps"] == so["ccd_clamps"]
        assert sg["iterations"] == so["iterations"]
        assert sg["intersections"] == oracle.count_intersections(osc, xo) == 0
        assert sg["uncertain"] == 0
        v = scenes.next_velocity(sc, xo, x)
        x, xt = xo, scenes.predict(sc, xo, v)
    gpu.close()


def test_validate_input_rejects_intersecting_start(cuda):
    sc = scenes.two_cloths(n=12, side=0.11, sep=0.002, omega=0.0, noise=0.0)
    x = sc.x0.copy()
    n = len(x) // 2
    x[n:] += np.array([0.0031, 0.0, 0.0017])  # off the bottom grid's lines
    # push one vertex of the top cloth 1 mm through the bottom cloth
    k = n + 5 * 12 + 5
    x[k, 1] = -0.001
    osc = oracle.OracleScene(sc)
    expected = oracle.count_intersections(osc, x)
    assert expected > 0
    gpu = cch.Scene(sc, cch.params_for(sc, validate_input=1))
    with pytest.raises(cch.CchError) as e:
        gpu.step(T(x, cuda), T(x, cuda))
    assert e.value.code == 7
    # the same scene accepts a feasible start
    x[k, 1] = 0.002
    out, st = gpu.step(T(x, cuda), T(x, cuda))
    assert st["iterations"] == 1
    gpu.close()


def test_acceptance_counts_match_oracle_on_intersecting_state(cuda):
    # with acceptance on, an infeasible start that does not move is reported
    sc = scenes.two_cloths(n=12, side=0.11, sep=0.002, omega=0.0, noise=0.0)
    x = sc.x0.copy()
    n = len(x) // 2
    x[n:] += np.array([0.0031, 0.0, 0.0017])
    for k in (n + 3 * 12 + 3, n + 7 * 12 + 8):
        x[k, 1] = -0.001
    osc = oracle.OracleScene(sc)
    expected = oracle.count_intersections(osc, x)
    im = sc.inv_mass.copy()
    im[:] = 0.0  # everything fixed: x^{t+1} = x^t
    sc.inv_mass = im
    gpu = cch.Scene(sc, cch.params_for(sc, accept_check=1))
    out, st = gpu.step(T(x, cuda), T(x, cuda))
    assert np.array_equal(out.cpu().numpy(), x)
    assert st["uncertain"] == 0
    assert st["intersections"] == expected
    gpu.close()


def test_non_finite_input_rejected(cuda):
    # a NaN or infinite coordinate is detected on the device: no iteration
    # runs and the call returns CCH_E_INVALID_ARG; the scene stays usable
    sc = scenes.two_cloths(n=12, side=0.11, sep=0.004, omega=3.0, noise=0.2, seed=6)
    x, xt, _ = scenes.initial(sc)
    gpu = cch.Scene(sc, cch.params_for(sc))
    for which, k, val in (("x_tilde", 7, np.nan), ("x_t", 30, np.inf), ("x_tilde", 100, -np.inf)):
        a, b = x.copy(), xt.copy()
        (b if which == "x_tilde" else a)[k, 1] = val
        with pytest.raises(cch.CchError) as e:
            gpu.step(T(a, cuda), T(b, cuda))
        assert e.value.code == 1, which
    out, st = gpu.step(T(x, cuda), T(xt, cuda))
    xo, so, _ = oracle.handle_step(oracle.OracleScene(sc), oracle.params_for(sc), x, xt)
    assert np.max(np.abs(out.cpu().numpy() - xo)) <= 1e-9 * max(1.0, np.max(np.abs(xo)))
    assert st["iterations"] == so["iterations"]
    gpu.close()
