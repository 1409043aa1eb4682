"""Pins of the oracle's Frogsort (Symmetric merging, Frogsort0 and Frogsort1
sections) against the paper's layout tables and its stated operation counts."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows, meta = [], {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line:
                continue
            if line.startswith("#"):
                if line.startswith("# params:"):
                    for part in line[len("# params:"):].split(","):
                        k, v = part.split("=")
                        meta[k.strip()] = int(v.strip().split()[0])
                continue
            rows.append(line.split()[1:])
    return meta, rows


def _letters(labels):
    return [chr(ord("A") + v - 1) if v > 0 else chr(ord("a") - v - 1) for v in labels]


@pytest.mark.parametrize("name", ["frogsort0_layout.txt", "frogsort1_layout.txt"])
def test_layout_tables(name):
    meta, rows = _read_golden(name)
    trace = oracle.frog_trace(meta["n_data"], meta["split_unit"])
    assert trace.shape[0] == len(rows)
    for got, want in zip(trace, rows):
        got = _letters(got.tolist())
        assert len(got) == len(want)
        for g, w in zip(got, want):
            if w != ".":
                assert g == w, (name, got, want)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 8, 31, 64, 100, 1000, 4097])
def test_buffer_is_half(n):
    # Frogsort1 rule 2: the buffer has N/2 (integer division) slots
    assert oracle.frog_buffer(n) == n // 2
    assert oracle.frog_trace(n, 1).shape[1] == n + n // 2 if n <= 1000 else True


def _inner_sizes(n):
    """Sum over internal nodes of the inner child's size, for the tree whose
    surplus element always goes to the outer child: inner child = floor(n/2)."""
    if n <= 1:
        return 0
    return n // 2 + _inner_sizes((n + 1) // 2) + _inner_sizes(n // 2)


@pytest.mark.parametrize("n", [2, 3, 16, 1000, 1 << 12, 5000])
def test_presorted_moves_half(n):
    """Symmetric merging on presorted data: moves and comparisons drop to the
    inner run of every merge (about 50% per level)."""
    keys = np.arange(n, dtype=np.float64)
    k, p, c = oracle.frogsort(keys, np.arange(n, dtype=np.uint32), return_counters=True)
    assert np.array_equal(p, np.arange(n))
    assert c["merge_moves"] == _inner_sizes(n)
    assert c["merge_compares"] == _inner_sizes(n)
    if n & (n - 1) == 0:
        levels = n.bit_length() - 1
        assert c["merge_moves"] == levels * n // 2


@pytest.mark.parametrize("k", [4, 10, 12])
def test_knuthsort_moves_full(k):
    """Nocopy alternation: one initial copy, then every level moves 100%."""
    n = 1 << k
    keys = np.random.default_rng(k).random(n)
    _, _, c = oracle.knuthsort(keys, None, return_counters=True)
    assert c["moves"] == (k + 1) * n


def test_frogsort_random_and_ties_agree_with_definition():
    rng = np.random.default_rng(3)
    for n in [2, 3, 9, 10, 255, 256, 257, 4099, 20000]:
        for keys in (rng.random(n), rng.integers(0, 4, n).astype(np.float64)):
            p = np.arange(n, dtype=np.uint32)
            want = oracle.stable_sort(keys, p)
            for unit in (1, 2):
                if unit == 2 and n % 2:
                    continue
                got = oracle.frogsort(keys, p, split_unit=unit)
                assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_frogsort0_needs_even():
    with pytest.raises(ValueError):
        oracle.frogsort(np.zeros(3), None, split_unit=2)
