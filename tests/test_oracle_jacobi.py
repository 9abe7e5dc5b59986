"""Closed-form pins of the oracle's projected Jacobi variant (Sec. 4.3.2).

Jacobi computes every multiplier change from the same y; constraint c is
under-relaxed by omega_c = omega / n_max(c), n_max(c) being the largest
number of constraints at a movable vertex of c.  These pins fix the parts
that a wrong implementation would change:
  * one constraint alone (n = 1): omega = 1 gives the Gauss-Seidel result
    exactly (so the update itself is Eq. LCP's), omega scales the move;
  * a chain of two stretched edges (n = 1, 2, 1): each edge is relaxed by
    omega / 2, both ends move by a quarter of omega times the excess, and the
    shared middle vertex stays put (Gauss-Seidel would move it), so the sum
    really is taken from one y;
  * two copies of one edge on a vertex pinned at the other end (n = 2): the
    excess obeys e_{s+1} = (1 - omega) e_s sweep after sweep, which holds
    only if the multipliers accumulate (lambda += omega_c dl); omega = 1.5
    overshoots, so every second sweep has dl < 0 and pulls back.
"""
from types import SimpleNamespace as NS

import numpy as np
import pytest

import oracle

U = np.array([0.6, 0.0, 0.8])
L0 = 0.02


def mini(inv_mass, tris=(), len_edges=(), points=()):
    inv_mass = np.asarray(inv_mass, float)
    return NS(n_verts=len(inv_mass), inv_mass=inv_mass, radius=None, tris=np.asarray(tris, np.int32).reshape(-1, 3),
              edges=np.zeros((0, 2), np.int32), len_edges=np.asarray(len_edges, np.int32).reshape(-1, 2),
              points=np.asarray(points, np.int32))


def jacobi(**kw):
    return oracle.params(solver=1, **kw)


@pytest.mark.parametrize("h", [0.2e-3, 0.7e-3])
def test_single_contact_omega_one_is_gauss_seidel(h):
    tri = np.array([[0.0, 0, 0], [1e-2, 0, 0], [0, 1e-2, 0]])
    x = np.vstack([[[2e-3, 3e-3, h]], tri])
    sc = mini([1.0, 0.0, 0.0, 0.0], tris=[[1, 2, 3]], points=[0])
    osc = oracle.OracleScene(sc)
    pgs = oracle.backward_once(osc, oracle.params(), x, x, x)
    jac = oracle.backward_once(osc, jacobi(jacobi_omega=1.0), x, x, x)
    assert np.array_equal(pgs, jac)
    assert abs(jac[0, 2] - 1e-3) <= 1e-15  # lifted to delta (P6)
    half = oracle.backward_once(osc, jacobi(jacobi_omega=0.5), x, x, x)
    assert abs(half[0, 2] - (h + 0.5 * (1e-3 - h))) <= 1e-15
    assert np.array_equal(half[1:], x[1:])


@pytest.mark.parametrize("omega", [0.5, 1.0])
@pytest.mark.parametrize("sigma", [1.1, 1.2])
def test_chain_moves_ends_not_middle(omega, sigma):
    y0 = np.array([0.0, 1.0, 2.0])[:, None] * L0 * U        # rest shape (target)
    y = np.array([0.0, 1.5, 3.0])[:, None] * L0 * U         # both edges at 1.5 L0
    sc = mini([1.0, 1.0, 1.0], len_edges=[[0, 1], [1, 2]])
    out = oracle.backward_once(oracle.OracleScene(sc), jacobi(sigma=sigma, jacobi_omega=omega), y0, y, y0)
    move = 0.25 * omega * (1.5 - sigma) * L0
    expect = np.array([move, 1.5 * L0, 3.0 * L0 - move])[:, None] * U
    assert np.max(np.abs(out - expect)) <= 1e-17
    # Gauss-Seidel differs: the middle vertex moves
    gs = oracle.backward_once(oracle.OracleScene(sc), oracle.params(sigma=sigma), y0, y, y0)
    assert np.linalg.norm(gs[1] - y[1]) > 1e-4 * L0


@pytest.mark.parametrize("omega,sweeps", [(0.5, 1), (0.5, 3), (1.0, 1), (1.0, 3), (1.5, 1), (1.5, 2), (1.5, 4),
                                          (0.3, 3)])
def test_duplicate_edge_excess_recurrence(omega, sweeps):
    sigma = 1.1
    y0 = np.array([[0.0, 0, 0], L0 * U])
    y = np.array([[0.0, 0, 0], 1.5 * L0 * U])
    sc = mini([0.0, 1.0], len_edges=[[0, 1], [0, 1]])
    prm = jacobi(sigma=sigma, jacobi_omega=omega, gs_sweeps=sweeps)
    out = oracle.backward_once(oracle.OracleScene(sc), prm, y0, y, y0)
    excess = (1.5 - sigma) * (1.0 - omega) ** sweeps
    assert np.array_equal(out[0], y[0])
    assert abs(np.linalg.norm(out[1]) - (sigma + excess) * L0) <= 1e-16
    assert np.allclose(np.cross(out[1], U), 0.0, atol=1e-17)
