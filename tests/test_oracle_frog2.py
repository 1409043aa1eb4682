"""Pins of the oracle's Frogsort2 (Frogsort2 section: imbalanced symmetric
merging, inner branch p, buffer floor(p n)): at p = 1/2 it is Frogsort1 move
for move (Frogsort1 is pinned by the paper's layout tables); for other p its
result is the stable sort (brute force over every small input in
test_oracle_bruteforce.py, NumPy's stable sort on larger ones here); its
buffer is floor(p n); on presorted input a merge moves only the inner run."""
import numpy as np
import pytest

import oracle

PS = [(1, 2), (1, 3), (1, 4), (1, 8), (3, 10), (1, 16)]


@pytest.mark.parametrize("n", [2, 3, 5, 8, 13, 64, 100, 1000, 4097])
def test_half_is_frogsort1(n):
    rng = np.random.default_rng(n)
    keys = rng.integers(0, max(2, n // 3), n).astype(np.float64)
    pay = np.arange(n, dtype=np.uint32)
    k1, p1, c1 = oracle.frogsort(keys, pay, return_counters=True)
    k2, p2, c2 = oracle.frogsort2(keys, pay, p_num=1, p_den=2, leaf=1, return_counters=True)
    assert np.array_equal(k1.view(np.uint64), k2.view(np.uint64)) and np.array_equal(p1, p2)
    assert c1 == c2                     # same moves and comparisons: the same algorithm
    assert oracle.frog2_buffer(n, 1, 2) == oracle.frog_buffer(n)


@pytest.mark.parametrize("p", PS)
@pytest.mark.parametrize("n", [777, 8192, 50000])
def test_random_matches_numpy(p, n):
    rng = np.random.default_rng(n + p[1])
    keys = rng.integers(0, n // 4, n).astype(np.float64)
    pay = np.arange(n, dtype=np.uint32)
    k, q = oracle.frogsort2(keys, pay, p_num=p[0], p_den=p[1], leaf=64)
    idx = np.argsort(keys, kind="stable")
    assert np.array_equal(k, keys[idx]) and np.array_equal(q, pay[idx])


@pytest.mark.parametrize("p", PS)
def test_buffer_is_floor_pn(p):
    for n in (1, 2, 7, 1000, 123457):
        assert oracle.frog2_buffer(n, *p) == (n * p[0]) // p[1]


def test_presorted_moves_only_inner_runs():
    """Ascending input, p = 1/4: a data-left node's outer (left) run is already
    in place and its inner run moves once; a data-right node mirrors it.  So the
    merge moves of a presorted input equal the sum over merged nodes of the
    inner child's size, and there are fewer of them than in Frogsort1."""
    n = 4096
    keys = np.arange(n, dtype=np.float64)
    _, _, c4 = oracle.frogsort2(keys, None, p_num=1, p_den=4, leaf=1, return_counters=True)
    _, _, c2 = oracle.frogsort2(keys, None, p_num=1, p_den=2, leaf=1, return_counters=True)
    # every element of an inner run moves exactly once per merge it takes part in
    assert 0 < c4["merge_moves"]
    # Frogsort1 moves n/2 per level, log2 n levels
    assert c2["merge_moves"] == (n // 2) * 12
    # with p = 1/4 each merge moves only a quarter of its node
    assert c4["merge_moves"] < c2["merge_moves"]
