"""The velocity filter of Sec. 6.3 (friction), a pre-pass on the
frictionless target before the collision-handling step (no GPU).

Pins:
* closest points on a triangle satisfy the optimality condition of a
  projection onto a convex set ((p - q).(v - q) <= 0 at the three corners),
  with non-negative weights that sum to 1;
* a vertex pushed into a fixed triangle: the normal correction restores the
  separation, and Coulomb's law reduces the tangential motion by mu times it,
  or stops it when mu is large (sticking); a separating or distant vertex
  keeps its target bitwise;
* the correction of a pair of free vertices conserves momentum;
* the kinematic rotation is a rigid rotation by |w| dt;
* on the oracle, a spinning sphere drags a resting cloth with friction and
  not without it, and every step stays intersection-free."""
import math

import numpy as np
import pytest

import oracle
from paper_2211_04045_gb300 import scenes as S


def test_closest_point_optimality():
    rng = np.random.default_rng(0)
    P, A, B, C = (rng.normal(size=(4000, 3)) for _ in range(4))
    w = S.closest_on_triangle(P, A, B, C)
    assert (w >= -1e-12).all() and np.abs(w.sum(1) - 1.0).max() < 1e-12
    q = w[:, :1] * A + w[:, 1:2] * B + w[:, 2:] * C
    scale = 1.0 + np.linalg.norm(P - q, axis=1)
    for V in (A, B, C):
        g = np.einsum("ij,ij->i", P - q, V - q)
        assert (g <= 1e-12 * scale * (1.0 + np.linalg.norm(V - q, axis=1))).all()


def plane_scene():
    # a large fixed triangle in the plane y = 0 and one free vertex above it
    x = np.array([[-1.0, 0.0, -1.0], [1.0, 0.0, -1.0], [0.0, 0.0, 1.0], [0.1, 0.0, 0.2]])
    im = np.array([0.0, 0.0, 0.0, 1.0])
    return x, im, np.array([[0, 1, 2]])


@pytest.mark.parametrize("mu", [0.5, 10.0])
def test_coulomb_closed_form(mu):
    x, im, t = plane_scene()
    d0, dn, dt_ = 0.8e-3, -0.5e-3, 1.0e-3   # separation, normal and tangential target motion
    x[3, 1] = d0
    y = x.copy()
    y[3] += [dt_, dn, 0.0]
    out = S.friction_filter(x, y, im, t, mu=mu, reach=2e-3, sep=1e-3)
    pen = 1e-3 - (d0 + dn)                   # 0.7 mm
    assert abs(out[3, 1] - 1e-3) < 1e-15      # the normal correction restores the separation
    slide = max(dt_ - mu * pen, 0.0)          # Coulomb: |friction| <= mu |normal correction|
    assert abs((out[3, 0] - x[3, 0]) - slide) < 1e-15
    assert abs(out[3, 2] - x[3, 2]) < 1e-15 and np.array_equal(out[:3], y[:3])


def test_separating_or_distant_vertex_keeps_its_target():
    x, im, t = plane_scene()
    for d0, dn in ((0.8e-3, 0.5e-3), (3e-3, -1e-3)):
        x[3, 1] = d0
        y = x.copy()
        y[3] += [1e-3, dn, -2e-3]
        assert np.array_equal(S.friction_filter(x, y, im, t, mu=0.5, reach=2e-3, sep=1e-3), y)


def test_free_pair_conserves_momentum():
    rng = np.random.default_rng(3)
    x = np.array([[0.0, 0.0, 0.0], [0.01, 0.0, 0.0], [0.0, 0.0, 0.01], [0.002, 0.0008, 0.003]])
    im = rng.uniform(0.5, 2.0, 4)
    y = x + rng.normal(0.0, 1e-3, x.shape)
    y[3, 1] = x[3, 1] - 1e-3
    out = S.friction_filter(x, y, im, np.array([[0, 1, 2]]), mu=0.4, reach=2e-3, sep=1e-3)
    assert not np.array_equal(out, y)
    mom = ((out - y) / im[:, None]).sum(0)
    assert np.abs(mom).max() < 1e-15


def test_rotation_is_rigid():
    p = np.array([[0.3, 0.1, 0.0], [0.0, -0.2, 0.4]])
    q = S.rotate(p, np.array([0.0, 0.5, 0.0]), np.zeros(3))
    assert np.allclose(np.linalg.norm(q, axis=1), np.linalg.norm(p, axis=1), rtol=0, atol=1e-15)
    # about +y by 0.5 rad: (x, z) -> (x cos + z sin, -x sin + z cos)
    assert np.allclose(q[0], [0.3 * math.cos(0.5), 0.1, -0.3 * math.sin(0.5)], atol=1e-16)


def cap_turn(x, x0, nc):
    top = np.linalg.norm(x0[:nc, [0, 2]], axis=1) < 0.08
    a = np.arctan2(x[:nc, 2], x[:nc, 0]) - np.arctan2(x0[:nc, 2], x0[:nc, 0])
    return float(np.mean(((a + np.pi) % (2 * np.pi) - np.pi)[top]))


def test_oracle_sphere_drags_the_cloth_with_friction():
    turns = {}
    for mu in (0.0, 0.5):
        sc = S.cloth_on_rotating_sphere(n=16, side=0.5, sphere_subdiv=2, sphere_r=0.15, omega=2.0, mu=mu)
        osc = oracle.OracleScene(sc)
        prm = oracle.params_for(sc)
        x, xt, v = S.initial(sc)
        x0 = x.copy()
        for _ in range(10):
            xn, st, _ = oracle.handle_step(osc, prm, x, xt)
            assert oracle.count_intersections(osc, xn) == 0
            # a step that runs to L is the stall of Eq. forward2 where a pair's
            # distance collapses: its vertices are held by the D_i floor
            assert st["converged"] == 1 or st["frozen_vertices"] > 0
            v = S.next_velocity(sc, xn, x)
            x, xt = xn, S.predict(sc, xn, v)
        turns[mu] = cap_turn(x, x0, 16 * 16)
    # the sphere turns by -0.67 rad about +y in these ten steps
    assert turns[0.5] < -0.1 and abs(turns[0.0]) < 0.05, turns


def test_torch_dynamics_rotates_the_kinematic_sphere_like_numpy():
    # the benchmark chain's GPU copy of the dynamics (here on the CPU): the
    # frictionless target with the sphere's scripted rotation equals numpy's
    import dataclasses
    import torch
    sc = S.cloth_on_rotating_sphere(n=16, side=0.5, sphere_subdiv=2, sphere_r=0.15, omega=2.0, mu=0.5)
    x, _, v = S.initial(sc)
    v = v + np.random.default_rng(2).normal(0.0, 0.1, size=v.shape)
    want = S.predict(dataclasses.replace(sc, friction=None), x, v)
    dyn = S.TorchDynamics(sc, torch.device("cpu"))
    got = dyn.predict_frictionless(torch.tensor(x), torch.tensor(v)).numpy()
    assert np.max(np.abs(got - want)) <= 1e-15
    with pytest.raises(NotImplementedError):
        dyn.predict(torch.tensor(x), torch.tensor(v))
