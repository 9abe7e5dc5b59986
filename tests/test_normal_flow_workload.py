"""The globally injective normal flow of Sec. 7.4 as a second workload (no
GPU).  Its target (Eq. normal flow) is an input of the collision-handling
step, produced by the seeded input generators; these tests pin that target
to closed forms, and check on the oracle that the step keeps the flow free
of self-intersections while the raw targets are not.

Pins:
* the cotangent Laplacian reproduces linear functions: zero at the interior
  vertices of a jittered planar grid;
* on a unit sphere it approaches the mean-curvature normal, Lap x = -2 n,
  with first-order convergence of the largest error (mixed Voronoi areas);
* area-weighted vertex normals match the analytic normals of a sphere and a
  torus, and point outward;
* without smoothing the target is x + sign beta n; the smoothing is
  invariant under translation;
* the torch version the benchmark chains with equals the numpy one."""
import numpy as np
import pytest

import oracle
from paper_2211_04045_gb300 import scenes as S


def test_cotan_laplacian_linear_precision():
    x, t = S.grid_cloth(9, 1.0, 0.0)
    rng = np.random.default_rng(0)
    interior = np.array([i * 9 + j for i in range(1, 8) for j in range(1, 8)])
    x[interior, 0] += rng.uniform(-0.02, 0.02, len(interior))
    x[interior, 2] += rng.uniform(-0.02, 0.02, len(interior))
    L = S.cotan_laplacian(x, t)
    assert np.abs(L[interior]).max() < 1e-12
    # a linear field (here the coordinates plus a linear function in y) is reproduced too
    x3 = x.copy()
    x3[:, 1] = 0.3 * x[:, 0] - 0.7 * x[:, 2]
    L3 = S.cotan_laplacian(x3, t)
    assert np.abs(L3[interior]).max() < 1e-12


def test_cotan_laplacian_sphere_mean_curvature():
    errs = []
    for sd in (2, 3, 4):
        x, t = S.icosphere(sd, 1.0)
        errs.append(float(np.linalg.norm(S.cotan_laplacian(x, t) + 2.0 * x, axis=1).max()))
    assert errs[-1] < 0.01
    for a, b in zip(errs, errs[1:]):
        assert b < 0.6 * a  # first order: the largest error halves with each subdivision
    # scaling: Lap x of a sphere of radius R is -2 n / R
    x, t = S.icosphere(4, 0.25)
    assert np.linalg.norm(S.cotan_laplacian(x, t) + 2.0 * x / 0.25 ** 2, axis=1).max() < 0.01 / 0.25


def test_vertex_normals_sphere_and_torus():
    x, t = S.icosphere(3, 2.0, center=(0.1, -0.2, 0.3))
    n = S.vertex_normals(x, t)
    radial = (x - np.array([0.1, -0.2, 0.3])) / 2.0
    assert (1.0 - np.einsum("ij,ij->i", n, radial)).max() < 1e-4
    R, r = 0.1, 0.02
    x, t = S.torus_mesh(64, 24, R, r)
    n = S.vertex_normals(x, t)
    u = np.arctan2(x[:, 1], x[:, 0])
    core = np.stack([R * np.cos(u), R * np.sin(u), np.zeros_like(u)], 1)
    na = (x - core) / r
    assert (1.0 - np.einsum("ij,ij->i", n, na)).max() < 1e-5
    assert np.allclose(np.linalg.norm(n, axis=1), 1.0, atol=1e-14)


def test_target_without_smoothing_and_translation_invariance():
    x, t = S.torus_mesh(32, 12, 0.05, 0.01)
    for sign in (-1.0, 1.0):
        y = S.normal_flow_target(x, t, beta=2e-3, alpha=1e-6, sign=sign, iters=0)
        assert np.array_equal(y, x + (sign * 2e-3) * S.vertex_normals(x, t))
    c = np.array([0.3, -1.2, 0.7])
    d = S.normal_flow_target(x + c, t, 2e-3, 1e-6, -1.0) - c - S.normal_flow_target(x, t, 2e-3, 1e-6, -1.0)
    assert np.abs(d).max() < 1e-12


def test_torch_target_equals_numpy():
    torch = pytest.importorskip("torch")
    sc = S.normal_flow_torus(n_major=40, n_minor=14, R=0.03, r=0.006, sign=-1.0)
    dyn = S.TorchDynamics(sc, "cpu")
    x = sc.x0 + np.random.default_rng(1).normal(0.0, 1e-4, sc.x0.shape)
    a = S.predict(sc, x, None)
    b = dyn.predict(torch.tensor(x), None).numpy()
    assert np.abs(a - b).max() <= 1e-15


def flow_cases():
    return {
        "shrink": lambda: S.normal_flow_torus(n_major=48, n_minor=16, R=0.03, r=0.006, sign=-1.0),
        "grow": lambda: S.normal_flow_torus(n_major=48, n_minor=16, R=0.015, r=0.01, sign=1.0),
    }


@pytest.mark.parametrize("name", list(flow_cases()))
def test_oracle_keeps_the_flow_injective(name):
    sc = flow_cases()[name]()
    osc = oracle.OracleScene(sc)
    prm = oracle.params_for(sc)
    x = sc.x0.copy()
    assert oracle.count_intersections(osc, x) == 0
    raw_hits = 0
    for _ in range(4):
        y = S.predict(sc, x, None)
        raw_hits += oracle.count_intersections(osc, y)
        x, st, _ = oracle.handle_step(osc, prm, x, y)
        assert st["converged"] == 1
        assert oracle.count_intersections(osc, x) == 0
    assert raw_hits > 0  # the flow alone self-intersects within four steps
