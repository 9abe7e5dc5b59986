"""P2: closed-form times of impact of the oracle's CCD (the comparison scheme
of Sec. 5.1, used here as the segment safety check)."""
import numpy as np
import pytest

import oracle

TRI = np.array([[0.0, 0, 0], [1.0, 0, 0], [0, 1.0, 0]])


@pytest.mark.parametrize("h,v", [(0.3, 1.0), (0.05, 0.2), (1e-3, 0.5), (0.5, 0.75)])
def test_vertex_onto_static_triangle(h, v):
    x0 = np.concatenate([[[0.2, 0.2, h]], TRI])
    x1 = x0.copy()
    x1[0, 2] -= v
    hit, toi = oracle.ccd(oracle.VT, x0, x1)
    assert hit and abs(toi - h / v) < 1e-9


@pytest.mark.parametrize("h,u,v", [(0.3, 0.2, 0.5), (0.1, 0.4, 0.4)])
def test_triangle_rising_to_falling_vertex(h, u, v):
    x0 = np.concatenate([[[0.25, 0.25, h]], TRI])
    x1 = x0.copy()
    x1[0, 2] -= v
    x1[1:, 2] += u
    hit, toi = oracle.ccd(oracle.VT, x0, x1)
    assert hit and abs(toi - h / (u + v)) < 1e-9


@pytest.mark.parametrize("h,v", [(0.2, 0.5), (0.01, 0.02)])
def test_edge_onto_crossing_edge(h, v):
    x0 = np.array([[-1.0, 0, h], [1.0, 0, h], [0, -1.0, 0], [0, 1.0, 0]])
    x1 = x0.copy()
    x1[:2, 2] -= v
    hit, toi = oracle.ccd(oracle.EE, x0, x1)
    assert hit and abs(toi - h / v) < 1e-9


def test_misses():
    # vertex outside the triangle's shadow
    x0 = np.concatenate([[[0.8, 0.8, 0.3]], TRI])
    x1 = x0.copy()
    x1[0, 2] -= 1.0
    assert oracle.ccd(oracle.VT, x0, x1) == (False, None)
    # vertex stops short
    x0 = np.concatenate([[[0.2, 0.2, 0.3]], TRI])
    x1 = x0.copy()
    x1[0, 2] -= 0.25
    assert oracle.ccd(oracle.VT, x0, x1) == (False, None)
    # edges pass beside each other
    x0 = np.array([[-1.0, 2.0, 0.2], [1.0, 2.0, 0.2], [0, -1.0, 0], [0, 1.0, 0]])
    x1 = x0.copy()
    x1[:2, 2] -= 0.5
    assert oracle.ccd(oracle.EE, x0, x1) == (False, None)


@pytest.mark.parametrize("d0,v,R", [(0.5, 1.0, 0.0), (0.5, 1.0, 0.1), (0.02, 0.05, 0.004)])
def test_spheres_meeting_head_on(d0, v, R):
    # two spheres of radii R/2 approaching at relative speed v: contact at (d0 - R)/v
    x0 = np.array([[0.0, 0, 0], [d0, 0, 0]])
    x1 = np.array([[0.5 * v, 0, 0], [d0 - 0.5 * v, 0, 0]])
    hit, toi = oracle.ccd(oracle.VV, x0, x1, [R / 2, R / 2])
    # contact is registered 1e-9 m early (the touch tolerance): 1e-9 / v in time
    assert hit and abs(toi - (d0 - R) / v) <= 1e-9 / v + 1e-12
    # moving apart from a separated start: no contact
    far = np.array([[0.0, 0, 0], [d0, 0, 0]])
    apart = np.array([[-0.5 * v, 0, 0], [d0 + 0.5 * v, 0, 0]])
    assert oracle.ccd(oracle.VV, far, apart, [R / 2, R / 2]) == (False, None)


# ---- the conservative CCD (an independent check of the one above) ----------
def tangential_case():
    # a = (0,0,0), c = (0,1,0) fixed, b(t) = (1, 0, -0.1 t), p(t) = (0.2 + 0.1 t,
    # 0.2, 0.0025 - 0.03 t): the coplanarity function is 0.01 (t - 0.5)^2,
    # a double root without a sign change, and at t = 0.5 p lies on the
    # triangle (inside its projection: 0.25 + 0.2 < 1)
    x0 = np.array([[0.2, 0.2, 0.0025], [0.0, 0, 0], [1.0, 0, 0], [0, 1.0, 0]])
    x1 = np.array([[0.3, 0.2, 0.0025 - 0.03], [0.0, 0, 0], [1.0, 0, -0.1], [0, 1.0, 0]])
    return x0, x1


def test_tangential_touch_at_a_double_root():
    x0, x1 = tangential_case()
    q = 0.5 * (x0 + x1)
    assert oracle.point_triangle_dist(*q) < 1e-15
    for t in (0.4999, 0.5001):
        q = x0 + t * (x1 - x0)
        # 0.01 (1e-4)^2 over the normal's length (1 + 0.05^2)^(1/2)
        assert abs(oracle.point_triangle_dist(*q) - 1e-10 / np.sqrt(1.0025)) < 1e-16
    assert oracle.ccd_conservative(oracle.VT, x0, x1)
    # the coplanarity-root CCD finds no sign change and misses the touch;
    # this is why the CCD-based step rule always runs the exact acceptance
    hit, _ = oracle.ccd(oracle.VT, x0, x1)
    assert not hit


@pytest.mark.parametrize("h", [0.3, 0.02, 1e-3])
def test_conservative_ccd_on_closed_forms(h):
    # a vertex falling onto the triangle reaches it
    x0 = np.concatenate([[[0.2, 0.2, h]], TRI])
    x1 = x0.copy()
    x1[0, 2] -= 2.0 * h
    assert oracle.ccd_conservative(oracle.VT, x0, x1)
    # stopping at h/2 above it: certainly more than h/4 apart, not 0.51 h
    x1[0, 2] = 0.5 * h
    assert not oracle.ccd_conservative(oracle.VT, x0, x1, tol=0.25 * h)
    assert oracle.ccd_conservative(oracle.VT, x0, x1, tol=0.51 * h)
    # an edge sweeping over a crossing edge at height h stays h apart (more than
    # h/2 certified, not 1.01 h)
    e0 = np.array([[-1.0, -0.5, h], [1.0, -0.5, h], [0, -1.0, 0], [0, 1.0, 0]])
    e1 = e0.copy()
    e1[:2, 1] += 1.0
    assert not oracle.ccd_conservative(oracle.EE, e0, e1, tol=0.5 * h)
    assert oracle.ccd_conservative(oracle.EE, e0, e1, tol=1.01 * h)
    # two spheres of radius 0.1 passing with centre distance 0.2 + h
    s0 = np.array([[-1.0, 0.2 + h, 0.0], [0.0, 0.0, 0.0]])
    s1 = s0 + np.array([[2.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    rho = np.array([0.1, 0.1])
    assert not oracle.ccd_conservative(oracle.VV, s0, s1, rho, tol=0.5 * h)
    assert oracle.ccd_conservative(oracle.VV, s0, s1, rho, tol=1.01 * h)
