"""Pins of the oracle on larger random inputs: invariants that hold at any size
and special cases that reduce to NumPy's stable sort (a library routine)."""
import numpy as np
import pytest

import oracle
from paper_2402_01816_gb300 import inputs


@pytest.mark.parametrize("n", [0, 1, 2, 1000, 4097, 1 << 16, 1 << 20])
def test_matches_numpy_stable_sort_int64(n):
    rng = np.random.default_rng(n)
    keys = rng.integers(-2**63, 2**63 - 1, n, dtype=np.int64, endpoint=True)
    keys[: n // 3] = keys[n // 2: n // 2 + n // 3] if n >= 6 else keys[: n // 3]
    perm = np.argsort(keys, kind="stable")
    k, p = oracle.stable_sort(keys, np.arange(n, dtype=np.uint32))
    assert np.array_equal(p, perm) and np.array_equal(k, keys[perm])
    if n <= 1 << 16:
        k2, p2 = oracle.knuthsort(keys, np.arange(n, dtype=np.uint32))
        assert np.array_equal(p2, perm)


@pytest.mark.parametrize("pattern", ["uniform", "ties", "permut", "asc_noise", "desc", "mixture"])
def test_matches_numpy_stable_sort_f64(pattern):
    """Finite keys without -0.0: NumPy's stable sort orders like the oracle."""
    n = 1 << 16
    keys = inputs.make_keys(pattern, n, seed=5)
    perm = np.argsort(keys, kind="stable")
    for fn in (oracle.stable_sort, oracle.knuthsort, oracle.frogsort):
        k, p = fn(keys, np.arange(n, dtype=np.uint32))
        assert np.array_equal(p, perm), fn.__name__


@pytest.mark.parametrize("n", [1, 7, 1000, 1 << 14])
def test_descending_with_ties(n):
    """DescLeft: keys non-increasing, equal keys in input order.  For int64 keys
    without the minimum value this is NumPy's stable sort of the negated keys."""
    rng = np.random.default_rng(11)
    keys = rng.integers(-50, 50, n).astype(np.int64)
    perm = np.argsort(-keys, kind="stable")
    for fn in (oracle.stable_sort, oracle.knuthsort, oracle.frogsort):
        k, p = fn(keys, np.arange(n, dtype=np.uint32), oracle.DESC)
        assert np.array_equal(p, perm), fn.__name__
    # it is not the reverse of the ascending sort when there are ties
    ka, pa = oracle.stable_sort(keys, np.arange(n, dtype=np.uint32), oracle.ASC)
    if n >= 1000:
        assert not np.array_equal(pa[::-1], perm)


def test_invariants_edge_keys():
    """Non-decreasing, multiset-equal, stable -- on keys with NaNs and zeros."""
    rng = np.random.default_rng(4)
    alpha = inputs.edge_alphabet()
    keys = alpha[rng.integers(0, alpha.size, 50000)]
    k, p = oracle.stable_sort(keys, np.arange(keys.size, dtype=np.uint32))
    kb = k.view(np.uint64)
    assert np.array_equal(kb, keys.view(np.uint64)[p])
    assert np.array_equal(np.sort(kb), np.sort(keys.view(np.uint64)))
    for i in range(0, keys.size - 1, 97):
        c = oracle.compare(int(kb[i]), int(kb[i + 1]), oracle.F64)
        assert c < 0 or (c == 0 and p[i] < p[i + 1])
    k2, p2 = oracle.knuthsort(keys, np.arange(keys.size, dtype=np.uint32))
    assert np.array_equal(p2, p)


def test_final_position_matches_sort():
    rng = np.random.default_rng(9)
    keys = rng.integers(0, 30, 3000).astype(np.float64)
    _, p = oracle.stable_sort(keys, np.arange(keys.size, dtype=np.uint32))
    where = np.empty_like(p)
    where[p] = np.arange(p.size, dtype=np.uint32)
    for i in rng.integers(0, keys.size, 40):
        assert oracle.final_position(keys, int(i)) == where[i]


def test_segmented_is_per_segment():
    keys, pay, off = inputs.segments(nseg=300, seed=2, median=40.0, hi=2000)
    k, p = oracle.segmented_sort(keys, pay, off)
    for s in range(off.size - 1):
        a, b = off[s], off[s + 1]
        perm = np.argsort(keys[a:b], kind="stable") + a
        assert np.array_equal(p[a:b], perm)
