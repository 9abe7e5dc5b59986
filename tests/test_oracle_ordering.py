"""Pins of the Gauss-Seidel sweep order of the oracle (Sec. 4.3, readings
R10 and R11).

The priorities come from SplitMix64, pinned to its published sequence.  The
sweep applies contacts before edge-length constraints (R10) and, within
each, constraints by descending priority splitmix64(seed ^ key) (R11).  Two
closed-form cases fix both rules: a chain of two stretched edges, whose
result depends on which edge goes first, and a point held by a contact and
an edge that pull it in opposite directions.
"""
from types import SimpleNamespace as NS

import numpy as np
import pytest

import oracle

EDGE_KIND = 3 << 62


def test_splitmix64_published_sequence():
    # first two outputs of SplitMix64 started from state 0
    assert oracle.splitmix64(0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4


def test_splitmix64_is_injective_on_keys():
    keys = np.arange(20000, dtype=np.uint64) | np.uint64(1 << 62)
    pr = {oracle.splitmix64(int(k) ^ 12345) for k in keys}
    assert len(pr) == len(keys)


def mini(inv_mass, len_edges=(), points=(), radius=None):
    inv_mass = np.asarray(inv_mass, float)
    return NS(n_verts=len(inv_mass), inv_mass=inv_mass, radius=None if radius is None else np.asarray(radius, float),
              tris=np.zeros((0, 3), np.int32), edges=np.zeros((0, 2), np.int32),
              len_edges=np.asarray(len_edges, np.int32).reshape(-1, 2), points=np.asarray(points, np.int32))


@pytest.mark.parametrize("seed", range(8))
def test_edges_swept_by_descending_priority(seed):
    # vertices 0-1-2 on a line, both edges at 1.5 L0, sigma = 1.1, unit masses.
    # The first edge applied moves each of its ends by 0.2 L0; the second then
    # sees 1.7 L0 and moves its ends by 0.3 L0.
    L0, u = 0.01, np.array([0.0, 0.6, 0.8])
    y0 = np.array([0.0, 1.0, 2.0])[:, None] * L0 * u
    y = np.array([0.0, 1.5, 3.0])[:, None] * L0 * u
    sc = mini([1.0, 1.0, 1.0], len_edges=[[0, 1], [1, 2]])
    out = oracle.backward_once(oracle.OracleScene(sc), oracle.params(seed=seed), y0, y, y0)
    p0, p1 = (oracle.splitmix64(seed ^ (EDGE_KIND | e)) for e in (0, 1))
    if p0 > p1:
        expect = [0.2, 1.6, 2.7]
    else:
        expect = [0.3, 1.4, 2.8]
    assert np.max(np.abs(out - np.array(expect)[:, None] * L0 * u)) <= 1e-17, (seed, p0 > p1)


def test_seeds_cover_both_orders():
    firsts = {oracle.splitmix64(s ^ EDGE_KIND) > oracle.splitmix64(s ^ (EDGE_KIND | 1)) for s in range(8)}
    assert firsts == {True, False}


def test_contacts_before_edges():
    # q (fixed point) at 0, p (movable point) at x = 0.5 mm, r (fixed) at
    # -5 mm; delta = 1 mm, zero radii.  The edge p-r has L0 = 5.5 mm and
    # sigma = 1.05, so it pulls p to -5 + 5.775 = 0.775 mm.  At the start
    # y_p = 2 mm, where the contact is satisfied.  Contacts first: the contact
    # does nothing, then the edge moves p to 0.775 mm (inside delta of q).
    # Edges first would end at 1 mm (the contact pushing p back out).
    mm = 1e-3
    e = np.array([0.0, 0.0, 1.0])
    x = np.array([0.0, 0.5, -5.0])[:, None] * mm * e
    y = np.array([0.0, 2.0, -5.0])[:, None] * mm * e
    sc = mini([0.0, 1.0, 0.0], len_edges=[[1, 2]], points=[0, 1], radius=[0.0, 0.0, 0.0])
    out = oracle.backward_once(oracle.OracleScene(sc), oracle.params(sigma=1.05, delta=1e-3), x, y, x)
    assert abs(out[1, 2] - 0.775 * mm) <= 1e-15
    assert np.array_equal(out[[0, 2]], y[[0, 2]])
