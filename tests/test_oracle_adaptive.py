"""Pins of the oracle's adaptive mergesorts against the operation counts the
paper states for them ("Full adaptivity", "Symmetric merging" and "Squidsort"
sections).  Their sorted results are pinned by brute force in
test_oracle_bruteforce.py; here the counters are pinned by closed forms and by
a plain recursion over the tree, written out independently of the oracle:

* Omitsort: presorted input costs one comparison per merge node (n - 1) and no
  move; strictly descending input cannot omit anything;
* Octosort: presorted, all-equal and strictly descending input cost n - 1
  comparisons and no move during the recursion; descending input is reversed
  once at the end;
* Geckosort1: one branch left-ascending, the other right-ascending, so about
  25% of the moves and comparisons are saved on ascending and on descending
  input alike (Frogsort1 saves 50% on ascending input only);
* Squidsort1: presorted, all-equal and strictly descending input cost one
  comparison per node ("0%") and move only the inner run of every merge
  ("50%"), plus one final reversal for descending input.
"""
import math

import numpy as np
import pytest

import oracle

SIZES = [2, 3, 5, 16, 100, 1000, 1 << 12, 5000]


def _check_sorted(fn, keys, order=oracle.ASC):
    k, p, c = fn(keys.copy(), np.arange(keys.size, dtype=np.uint32), order, return_counters=True)
    wk, wp = oracle.stable_sort(keys, np.arange(keys.size, dtype=np.uint32), order)
    assert np.array_equal(k.view(np.uint64), wk.view(np.uint64)) and np.array_equal(p, wp)
    return c


# ---------------------------------------------------------------- Omitsort / Octosort
@pytest.mark.parametrize("n", SIZES)
def test_omitsort_presorted_costs_no_move(n):
    """The merge reports where the data lies; non-overlapping halves are left
    where they are: n - 1 comparisons (one per merge node), no move at all."""
    c = _check_sorted(oracle.omitsort, np.arange(n, dtype=np.float64))
    assert c["moves"] == 0 and c["compares"] == n - 1


@pytest.mark.parametrize("k", [1, 2, 3, 6, 10, 12])
def test_omitsort_descending_merges_everything(k):
    """Strictly descending input, n = 2^k: every node's halves overlap in the
    target order, so each level moves all n elements and the data ends in the
    buffer after an odd number of levels (one copy back).  Each merge takes
    the right run first: nr comparisons, plus the node's non-overlap test."""
    n = 1 << k
    c = _check_sorted(oracle.omitsort, np.arange(n, 0, -1, dtype=np.float64))
    assert c["moves"] == k * n + (n if k % 2 else 0)
    assert c["compares"] == k * n // 2 + (n - 1)


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("pattern", ["asc", "ties", "desc"])
def test_octosort_bi_adaptive(n, pattern):
    """Octosort's order is decided by the data: presorted, all-equal and
    strictly descending input need one comparison per merge node and no move
    during the recursion; descending input is reversed once at the end
    (floor(n/2) swaps, two moves each)."""
    keys = {"asc": np.arange(n, dtype=np.float64), "ties": np.full(n, 7.0),
            "desc": np.arange(n, 0, -1, dtype=np.float64)}[pattern]
    c = _check_sorted(oracle.octosort, keys)
    assert c["compares"] == n - 1
    assert c["moves"] == (2 * (n // 2) if pattern == "desc" else 0)


@pytest.mark.parametrize("n", [16, 1000, 4096])
def test_octosort_descending_order_is_the_mirror_case(n):
    """Sorting ascending input in descending order is Octosort's reversal case."""
    c = _check_sorted(oracle.octosort, np.arange(n, dtype=np.float64), oracle.DESC)
    assert c["compares"] == n - 1 and c["moves"] == 2 * (n // 2)


@pytest.mark.parametrize("seed", range(4))
def test_omit_and_octo_on_random_input_do_real_work(seed):
    """On random input neither can omit much: each moves at least n log2(n) / 2
    elements, and no comparison sort gets by with fewer than log2(n!)
    comparisons on average (a few below it on a single input)."""
    n = 1 << 12
    keys = np.random.default_rng(70 + seed).random(n)
    bound = math.lgamma(n + 1) / math.log(2)
    for fn in (oracle.omitsort, oracle.octosort):
        c = _check_sorted(fn, keys)
        assert c["moves"] >= 12 * n // 2 and c["compares"] >= 0.99 * bound


# ---------------------------------------------------------------- Geckosort1 / Squidsort1
def _tree_counts(n, side, rule):
    """Plain recursion over Frogsort1's tree (the outer child takes the surplus
    element: inner child floor(n/2)); rule(n, side, n_inner) gives a merge
    node's (moves, comparisons)."""
    if n <= 1:
        return 0, 0
    nin = n // 2
    nout = n - nin
    left, right = ((nout, 0), (nin, 1)) if side == 0 else ((nin, 0), (nout, 1))
    m0, c0 = rule(n, side, nin)
    m1, c1 = _tree_counts(*left, rule)
    m2, c2 = _tree_counts(*right, rule)
    return m0 + m1 + m2, c0 + c1 + c2


def _gecko_asc(n, side, nin):
    # data-left nodes are left-ascending: the inner (right) run comes first and
    # ends the merge; data-right nodes are right-ascending: everything moves
    return (nin, nin) if side == 0 else (n, n - nin)


def _gecko_desc(n, side, nin):
    return (n, n - nin) if side == 0 else (nin, nin)


@pytest.mark.parametrize("n", SIZES)
def test_geckosort_adaptive_both_ways(n):
    for keys, rule in ((np.arange(n, dtype=np.float64), _gecko_asc),
                       (np.arange(n, 0, -1, dtype=np.float64), _gecko_desc)):
        c = _check_sorted(oracle.geckosort, keys)
        moves, compares = _tree_counts(n, 0, rule)
        assert c["merge_moves"] == moves and c["compares"] == compares


@pytest.mark.parametrize("k", [10, 12, 14])
def test_geckosort_saves_a_quarter_on_both_orders(k):
    """n = 2^k: below the root, half of every level's elements lie in data-left
    nodes (saving half of their moves) and half in data-right nodes (saving
    none) on ascending input, and the other way round on descending input: a
    quarter of the moves of a full merge per level either way."""
    n = 1 << k
    full = k * n
    for keys in (np.arange(n, dtype=np.float64), np.arange(n, 0, -1, dtype=np.float64)):
        c = _check_sorted(oracle.geckosort, keys)
        frac = c["merge_moves"] / full
        assert abs(frac - 0.75) < 0.5 / k + 1e-12, frac
    # Frogsort1, for contrast: half the moves on ascending input, all on descending
    _, _, fa = oracle.frogsort(np.arange(n, dtype=np.float64), None, return_counters=True)
    assert fa["merge_moves"] == full // 2


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("pattern", ["asc", "ties", "desc"])
def test_squidsort_presorted_zero_compares_half_moves(n, pattern):
    keys = {"asc": np.arange(n, dtype=np.float64), "ties": np.full(n, -3.5),
            "desc": np.arange(n, 0, -1, dtype=np.float64)}[pattern]
    c = _check_sorted(oracle.squidsort, keys)
    half, _ = _tree_counts(n, 0, lambda m, side, nin: (nin, 0))
    assert c["compares"] == n - 1
    assert c["merge_moves"] == half + (2 * (n // 2) if pattern == "desc" else 0)


@pytest.mark.parametrize("seed", range(3))
def test_symmetric_sorts_random_input_setup_matches_frogsort(seed):
    """Geckosort1 and Squidsort1 keep Frogsort1's layout: the same setup moves,
    and on random input a full merge's worth of work per level."""
    n = 5000
    keys = np.random.default_rng(80 + seed).random(n)
    _, _, f = oracle.frogsort(keys, None, return_counters=True)
    for fn in (oracle.geckosort, oracle.squidsort):
        c = _check_sorted(fn, keys)
        assert c["setup_moves"] == f["setup_moves"]
        assert c["merge_moves"] >= 0.9 * f["merge_moves"]
