"""The sampled proximity-set check used at full size (pair_sampling.py)
agrees with the oracle's whole-scene search on a scene small enough for it:
given the oracle's own P it passes, and it catches a dropped pair, an extra
pair and a wrong distance."""
import numpy as np
import pytest

import oracle
from paper_2211_04045_gb300 import scenes

from pair_sampling import check_sampled_pairs, jittered


@pytest.fixture(scope="module")
def case():
    sc = scenes.hair_sand(n_strands=200, segs=16, n_points=2000, grain_r=0.002, bowl_r=0.15, bowl_subdiv=3,
                          seg_len=0.005, seed=3)
    x0, xt, _ = scenes.initial(sc)
    x = jittered(sc, x0, 0.0015, 7)
    D = oracle.params_for(sc).d_max
    k, d = oracle.proximity(oracle.OracleScene(sc), x, D, mode=0, x_tilde=xt)
    return sc, x, xt, D, dict(zip(k.tolist(), d.tolist()))


def test_sampled_check_accepts_the_oracle_set(case):
    sc, x, xt, D, got = case
    assert check_sampled_pairs(sc, x, xt, D, got, 10**6, seed=1) >= len(got) // 2


@pytest.mark.parametrize("mistake", ["drop", "extra", "distance"])
def test_sampled_check_catches_mistakes(case, mistake):
    sc, x, xt, D, got = case
    bad = dict(got)
    k = sorted(bad)[len(bad) // 2]
    if mistake == "drop":
        del bad[k]
    elif mistake == "extra":
        bad[(1 << 62) | (5 << 31) | 7] = 0.0
    else:
        bad[k] = bad[k] + 1e-9
    with pytest.raises(AssertionError):
        check_sampled_pairs(sc, x, xt, D, bad, 10**6, seed=1)
