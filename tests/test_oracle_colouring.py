"""Pins of the randomized constraint colouring (Sec. 4.3, reading R11)."""
import numpy as np
import pytest

import oracle


def test_splitmix64_published_sequence():
    # first two outputs of SplitMix64 started from state 0
    assert oracle.splitmix64(0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4


def test_splitmix64_is_injective_on_keys():
    keys = np.arange(20000, dtype=np.uint64) | np.uint64(1 << 62)
    pr = {oracle.splitmix64(int(k) ^ 12345) for k in keys}
    assert len(pr) == len(keys)


@pytest.mark.parametrize("seed", range(12))
def test_greedy_colouring_valid_and_greedy(seed):
    rng = np.random.default_rng(seed)
    nvert = 60
    n = 200
    nv = rng.choice([2, 4], size=n).astype(np.int32)
    verts = np.full((n, 4), -1, np.int32)
    for i in range(n):
        verts[i, :nv[i]] = rng.choice(nvert, size=nv[i], replace=False)
    movable = (rng.uniform(size=nvert) > 0.15).astype(np.uint8)
    key = rng.permutation(n).astype(np.uint64) + np.uint64(7)
    prio = np.array([oracle.splitmix64(int(k) ^ 99) for k in key], dtype=np.uint64)
    ncol, col = oracle.colour_greedy(verts, nv, movable, prio, key)
    assert ncol == col.max() + 1

    def mv(i):
        return {int(v) for v in verts[i, :nv[i]] if movable[v]}

    order = sorted(range(n), key=lambda i: (int(prio[i]), int(key[i])), reverse=True)
    rank = {c: r for r, c in enumerate(order)}
    for i in range(n):
        higher = [j for j in range(n) if j != i and mv(i) & mv(j) and rank[j] < rank[i]]
        used = {int(col[j]) for j in higher}
        # valid: no conflict with any neighbour; greedy: smallest unused colour
        for j in range(n):
            if j != i and mv(i) & mv(j):
                assert col[i] != col[j]
        smallest = 0
        while smallest in used:
            smallest += 1
        assert col[i] == smallest
