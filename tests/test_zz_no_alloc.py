"""The allocation-free proximity query against the allocating one.

cch_query_pairs_noalloc serves callers that may not allocate device memory
while they run (real-time loops that reserve all of their memory up front,
hosts whose own memory manager forbids cudaMalloc).  It must return exactly
what cch_query_pairs returns, on consecutive calls that reuse its fixed
scratch array, refuse results larger than that array, and report an unknown
count (-1) when the scene's own pair buffers are too small for the query.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2211_04045_gb300 import cch, scenes

pytestmark = pytest.mark.gpu


def T(a, dev):
    import torch
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)


def test_noalloc_query_matches_allocating_query(cuda):
    sc = scenes.two_cloths(n=40, side=0.4, sep=0.004, omega=6.0, noise=0.3, seed=11)
    x0, xt, _ = scenes.initial(sc)
    gpu = cch.Scene(sc, cch.params_for(sc))
    rng = np.random.default_rng(12)
    # two calls in a row with different states and both query kinds; the
    # second call finds the first call's contents in the shared array
    cases = [(x0, 4e-3, True), (x0 + rng.normal(0.0, 0.002, size=x0.shape), 6e-3, False)]
    for x, D, cand in cases:
        k_ref, d_ref = gpu.query_pairs(T(x, cuda), T(xt, cuda), D, candidates=cand)
        k_new, d_new = gpu.query_pairs_noalloc(T(x, cuda), T(xt, cuda), D, candidates=cand)
        assert len(k_ref) > 0
        assert np.array_equal(k_new, k_ref)
        assert np.array_equal(d_new, d_ref)
    gpu.close()


def test_noalloc_query_rejects_results_beyond_its_array(cuda):
    sc = scenes.two_cloths(n=64, side=0.3, sep=0.004, omega=0.0, noise=0.0)
    x0 = sc.x0
    gpu = cch.Scene(sc, cch.params_for(sc))
    with pytest.raises(cch.CchError) as e:
        gpu.query_pairs_noalloc(T(x0, cuda), T(x0, cuda), 0.05, candidates=True)
    assert e.value.code == 5
    # a query that fits in the array still works afterwards
    k_ref, _ = gpu.query_pairs(T(x0, cuda), T(x0, cuda), 2e-3, candidates=True)
    k_new, _ = gpu.query_pairs_noalloc(T(x0, cuda), T(x0, cuda), 2e-3, candidates=True)
    assert 0 < len(k_ref) <= cch.Scene.NOALLOC_MAX_PAIRS
    assert np.array_equal(k_new, k_ref)
    gpu.close()


def test_noalloc_query_reports_unknown_count_when_scene_buffers_overflow(cuda):
    # a scene created with tiny pair buffers: the proximity query's FP32-filter
    # survivors (some 68,000 pairs within 6 mm) pass through them; the
    # allocating query grows them, the allocation-free one cannot, and says
    # that its count is unknown
    sc = scenes.two_cloths(n=40, side=0.4, sep=0.004, omega=6.0, noise=0.3, seed=11)
    x0, xt, _ = scenes.initial(sc)
    gpu = cch.Scene(sc, cch.params_for(sc, pair_capacity=64))
    xg, xtg = T(x0, cuda), T(xt, cuda)
    cnt = C.c_int64(12345)
    rc = cch.lib().cch_query_pairs_noalloc(gpu.h, C.c_void_p(xg.data_ptr()), C.c_void_p(xtg.data_ptr()), 6e-3, 0,
                                           None, None, 0, C.byref(cnt))
    assert rc == 5 and cnt.value == -1
    # the allocating query grows the buffers; afterwards both agree
    k_ref, d_ref = gpu.query_pairs(xg, xtg, 6e-3, candidates=False)
    k_new, d_new = gpu.query_pairs_noalloc(xg, xtg, 6e-3, candidates=False)
    assert 64 < len(k_ref) <= cch.Scene.NOALLOC_MAX_PAIRS
    assert np.array_equal(k_new, k_ref) and np.array_equal(d_new, d_ref)
    gpu.close()
