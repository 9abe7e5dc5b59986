"""The two pre-pass kernels against the numpy input generator, element by
element (1e-12 relative to the coordinates' scale):

- the target of the normal flow (Sec. 7.4, Eq. normal flow: area-weighted
  vertex normals, then Jacobi steps of the cotangent Laplacian with mixed
  Voronoi areas) on both torus cases, with 0 to 3 smoothing steps, at the
  initial surface and at perturbed ones;
- the friction velocity filter (Sec. 6.3) on the rotating-sphere scene, with
  the cloth draped into reach of the sphere and seeded perturbations of the
  positions and of the frictionless target, for sticking and sliding values
  of mu.

Both kernels are gathers in a fixed order, so a repeated call is bitwise
identical.
"""
import dataclasses

import numpy as np
import pytest

from paper_2211_04045_gb300 import cch, scenes

pytestmark = pytest.mark.gpu


def T(a, dev):
    import torch
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)


TORI = {
    "shrink": lambda: scenes.normal_flow_torus(n_major=96, n_minor=24, R=0.03, r=0.006, sign=-1.0),
    "grow": lambda: scenes.normal_flow_torus(n_major=96, n_minor=24, R=0.015, r=0.01, sign=1.0),
}


@pytest.mark.parametrize("name", list(TORI))
@pytest.mark.parametrize("iters", [0, 1, 3])
def test_normal_flow_target_matches_generator(cuda, name, iters):
    sc = TORI[name]()
    fl = dict(sc.flow, iters=iters)
    gpu = cch.Scene(sc, cch.params_for(sc))
    rng = np.random.default_rng(3)
    for k, x in enumerate([sc.x0, sc.x0 + rng.normal(0.0, 2e-4, size=sc.x0.shape)]):
        want = scenes.normal_flow_target(x, sc.tris, **fl)
        got = gpu.normal_flow_target(T(x, cuda), fl["beta"], fl["alpha"], fl["sign"], iters).cpu().numpy()
        scale = float(np.max(np.abs(want)))
        assert float(np.max(np.abs(got - want))) <= 1e-12 * scale, (name, iters, k)
        again = gpu.normal_flow_target(T(x, cuda), fl["beta"], fl["alpha"], fl["sign"], iters).cpu().numpy()
        assert np.array_equal(got, again)
    gpu.close()


def rotating_case(mu, seed):
    sc = scenes.cloth_on_rotating_sphere(n=16, side=0.5, sphere_subdiv=2, sphere_r=0.15, omega=2.0, mu=mu)
    rng = np.random.default_rng(seed)
    nc = 16 * 16
    x = sc.x0.copy()
    # the cloth draped 0.5 mm above the sphere where it lies over it
    r2 = x[:nc, 0] ** 2 + x[:nc, 2] ** 2
    over = r2 < 0.15 ** 2
    x[:nc, 1] = np.where(over, np.sqrt(np.maximum(0.15 ** 2 - r2, 0.0)) + 0.0005, x[:nc, 1])
    x[:nc] += rng.normal(0.0, 1e-4, size=(nc, 3))
    v = np.zeros_like(x)
    v[:nc] = rng.normal(0.0, 0.05, size=(nc, 3))
    v[:nc, 1] -= 0.1                          # pressed onto the sphere
    frictionless = dataclasses.replace(sc, friction=None)
    y = scenes.predict(frictionless, x, v)
    return sc, x, y


@pytest.mark.parametrize("mu", [0.1, 0.5, 2.0])
@pytest.mark.parametrize("seed", [0, 1])
def test_friction_filter_matches_generator(cuda, mu, seed):
    sc, x, y = rotating_case(mu, seed)
    f = sc.friction
    want = scenes.friction_filter(x, y, sc.inv_mass, sc.tris, **f)
    assert np.count_nonzero(np.any(want != y, axis=1)) > 10   # the filter acts on this state
    gpu = cch.Scene(sc, cch.params_for(sc))
    got = gpu.friction_filter(T(x, cuda), T(y, cuda), f["mu"], f["reach"], f["sep"]).cpu().numpy()
    scale = float(np.max(np.abs(want)))
    assert float(np.max(np.abs(got - want))) <= 1e-12 * scale, (mu, seed)
    # in place (y_out aliasing y) and repeated: bitwise the same
    yt = T(y, cuda)
    gpu.friction_filter(T(x, cuda), yt, f["mu"], f["reach"], f["sep"], out=yt)
    assert np.array_equal(yt.cpu().numpy(), got)
    gpu.close()


def test_friction_filter_keeps_far_targets(cuda):
    # the cloth 2 cm above the sphere: nothing within reach, y unchanged bitwise
    sc = scenes.cloth_on_rotating_sphere(n=16, side=0.5, sphere_subdiv=2, sphere_r=0.15, omega=2.0, mu=0.5,
                                         gap=0.02)
    x = sc.x0
    y = x + np.random.default_rng(1).normal(0.0, 1e-3, size=x.shape)
    gpu = cch.Scene(sc, cch.params_for(sc))
    got = gpu.friction_filter(T(x, cuda), T(y, cuda), 0.5, 2e-3, 1e-3).cpu().numpy()
    assert np.array_equal(got, y)
    gpu.close()
