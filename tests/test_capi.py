"""The C ABI without a GPU: the library loads, exports every function that
include/cch.h declares, fills Table 2's defaults, and rejects invalid
arguments before any device work."""
import ctypes as C
import os
import re
from types import SimpleNamespace as NS

import numpy as np
import pytest

from paper_2211_04045_gb300 import cch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    with open(os.path.join(ROOT, "include", "cch.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_]+\*?\s+\**(cch_[a-z_0-9]+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_symbol():
    names = declared_functions()
    assert len(names) >= 15
    lib = C.CDLL(cch.lib_path() if os.path.exists(cch.lib_path()) else cch.lib()._name)
    for n in names:
        assert hasattr(lib, n), n


def test_defaults_are_table_2():
    p = cch.params()
    assert (p.d_min, p.d_max, p.delta, p.sigma, p.gamma, p.eps) == (2e-3, 4e-3, 1e-3, 1.1, 0.9, 1e-4)
    assert p.max_iters == 2048 and p.gs_sweeps == 1
    # the step rule and CCD rounds agree with the oracle's defaults
    import oracle
    o = oracle.params()
    assert (p.step_rule, p.ccd_rounds, p.ccd_check) == (o.step_rule, o.ccd_rounds, o.ccd_check) == (0, 8, 0)


def topo(**kw):
    base = dict(n_verts=4, inv_mass=np.ones(4), radius=None, tris=np.array([[0, 1, 2]], np.int32),
                edges=np.zeros((0, 2), np.int32), len_edges=np.array([[0, 1]], np.int32),
                points=np.array([3], np.int32))
    base.update(kw)
    return NS(**base)


@pytest.mark.parametrize("bad", [
    dict(tris=np.array([[0, 1, 7]], np.int32)),          # index out of range
    dict(tris=np.array([[0, 1, 1]], np.int32)),          # repeated vertex
    dict(edges=np.array([[2, 2]], np.int32)),            # degenerate edge
    dict(len_edges=np.array([[0, -1]], np.int32)),       # negative index
    dict(points=np.array([4], np.int32)),                # point out of range
    dict(inv_mass=np.array([1.0, np.nan, 1.0, 1.0])),    # non-finite mass
    dict(inv_mass=np.array([1.0, -1.0, 1.0, 1.0])),      # negative mass
    dict(radius=np.array([0.0, 0.0, 0.0, -1e-3])),       # negative radius
])
def test_invalid_topology_rejected(bad):
    with pytest.raises(cch.CchError) as e:
        cch.Scene(topo(**bad), cch.params(), stream=0)
    assert e.value.code == 1


@pytest.mark.parametrize("field,value", [("d_min", 0.0), ("d_max", 1e-3), ("delta", 3e-3), ("gamma", 1.0),
                                         ("gs_sweeps", 0), ("precision", 7), ("solver", 3), ("max_iters", -1),
                                         ("constraint_form", 2), ("step_rule", 2), ("ccd_rounds", -1),
                                         ("ccd_rounds", 65)])
def test_invalid_params_rejected(field, value):
    p = cch.params()
    setattr(p, field, value)
    with pytest.raises(cch.CchError) as e:
        cch.Scene(topo(), p, stream=0)
    assert e.value.code == 1


def test_status_strings():
    L = cch.lib()
    for code in range(10):
        assert L.cch_status_string(code)


def test_server_admission_by_budget():
    # the budget check happens before any device work
    sv = cch.Server(1 << 20, cch.params(), max_active=2, stream=0)
    big = topo(n_verts=200000, inv_mass=np.ones(200000), len_edges=np.zeros((0, 2), np.int32),
               points=np.zeros(0, np.int32))
    with pytest.raises(cch.CchError) as e:
        sv.add_scene(big)
    assert e.value.code == 3
    sv.close()


@pytest.mark.parametrize("field,value", [("d_min", 0.0), ("delta", 3e-3), ("gamma", 1.0), ("max_iters", -1)])
def test_invalid_scene_params_rejected(field, value):
    # per-scene physical parameters are validated like the pool's, before
    # any device work, in batches and in the server
    good, bad = cch.params(), cch.params()
    setattr(bad, field, value)
    with pytest.raises(cch.CchError) as e:
        cch.Scene([topo(), topo()], cch.params(), stream=0, scene_params=[good, bad])
    assert e.value.code == 1
    with pytest.raises(ValueError):
        cch.Scene([topo(), topo()], cch.params(), stream=0, scene_params=[good])
    sv = cch.Server(1 << 20, cch.params(), max_active=2, stream=0)
    with pytest.raises(cch.CchError) as e:
        sv.add_scene(topo(), bad)
    assert e.value.code == 1
    sv.close()
