"""Brute-force pins of the oracle's sorts against the definition of a stable
sort (Definition of sorting chapter: AscLeft / DescLeft -- keys in order, equal
keys in input order).  For tiny n every permutation is enumerated and exactly
one must satisfy the definition; for n <= 8 every arrangement of a multiset is
checked against the definition's two conditions."""
import itertools

import numpy as np
import pytest

import oracle
from tests._orderfacts import f64_cmp, i64_cmp

ALPHABETS = [
    np.array([-0.0, 0.0, 1.0]),
    np.array([0x7ff8000000000000, 0xfff0000000000000, 0xfff8000000000001],
             dtype=np.uint64).view(np.float64),   # +NaN, -inf, -NaN
    np.array([np.inf, -np.inf, 2.5]),
]


def _cmp(a, b, order):
    c = f64_cmp(int(np.float64(a).view(np.uint64)), int(np.float64(b).view(np.uint64)))
    return -c if order == oracle.DESC else c


def _satisfies_definition(inp, perm, order):
    for x, y in zip(perm[:-1], perm[1:]):
        c = _cmp(inp[x], inp[y], order)
        if c > 0 or (c == 0 and x > y):
            return False
    return True


SORTS = {
    "definition": lambda k, p, o: oracle.stable_sort(k, p, o),
    "knuthsort": lambda k, p, o: oracle.knuthsort(k, p, o),
    "frogsort1": lambda k, p, o: oracle.frogsort(k, p, o, split_unit=1),
    "frogsort2_1/4": lambda k, p, o: oracle.frogsort2(k, p, o, p_num=1, p_den=4, leaf=1),
    "frogsort2_1/3_leaf2": lambda k, p, o: oracle.frogsort2(k, p, o, p_num=1, p_den=3, leaf=2),
    "frogsort2_1/8": lambda k, p, o: oracle.frogsort2(k, p, o, p_num=1, p_den=8, leaf=1),
    "omitsort": lambda k, p, o: oracle.omitsort(k, p, o),
    "octosort": lambda k, p, o: oracle.octosort(k, p, o),
    "geckosort1": lambda k, p, o: oracle.geckosort(k, p, o),
    "squidsort1": lambda k, p, o: oracle.squidsort(k, p, o),
}


@pytest.mark.parametrize("order", [oracle.ASC, oracle.DESC])
@pytest.mark.parametrize("alpha", range(len(ALPHABETS)))
def test_all_permutations_small(order, alpha):
    """n <= 5, every key sequence over a 3-letter alphabet: enumerate all n!
    index permutations; exactly one meets the definition, and every oracle
    sort returns it (payload = input index, keys bit-identical)."""
    letters = ALPHABETS[alpha]
    for n in range(0, 6):
        for seq in itertools.product(range(3), repeat=n):
            inp = letters[list(seq)] if n else np.zeros(0)
            ok = [p for p in itertools.permutations(range(n))
                  if _satisfies_definition(inp, p, order)]
            assert len(ok) == 1
            want = np.array(ok[0], dtype=np.uint32)
            for name, fn in SORTS.items():
                k, p = fn(inp, np.arange(n, dtype=np.uint32), order)
                assert np.array_equal(p, want), (name, seq)
                assert np.array_equal(k.view(np.uint64), inp[want].view(np.uint64)), name


@pytest.mark.parametrize("order", [oracle.ASC, oracle.DESC])
def test_multiset_arrangements_n8(order):
    """All distinct arrangements of an 8-key multiset with ties, signed zeros,
    infinities and NaNs: every oracle sort meets the definition."""
    ms = np.array([0x7ff8000000000000, 0xfff0000000000000, 0x8000000000000000, 0,
                   0x3ff0000000000000, 0x3ff0000000000000, 0x7ff0000000000000,
                   0xfff8000000000000], dtype=np.uint64).view(np.float64)
    seen = set()
    for perm in itertools.permutations(range(8)):
        inp = ms[list(perm)]
        key = inp.view(np.uint64).tobytes()
        if key in seen:
            continue
        seen.add(key)
        for name, fn in SORTS.items():
            k, p = fn(inp, np.arange(8, dtype=np.uint32), order)
            assert sorted(p.tolist()) == list(range(8)), name
            assert np.array_equal(k.view(np.uint64), inp[p].view(np.uint64)), name
            assert _satisfies_definition(inp, p.tolist(), order), (name, perm)
    assert len(seen) == 20160


def test_int64_small_exhaustive():
    vals = np.array([-2**63, -1, 0, 2**63 - 1], dtype=np.int64)
    for n in range(0, 6):
        for seq in itertools.product(range(4), repeat=n):
            inp = vals[list(seq)] if n else np.zeros(0, dtype=np.int64)
            for order in (oracle.ASC, oracle.DESC):
                for name, fn in SORTS.items():
                    k, p = fn(inp, np.arange(n, dtype=np.uint32), order)
                    for x, y in zip(p[:-1].tolist(), p[1:].tolist()):
                        c = i64_cmp(int(inp[x]), int(inp[y]))
                        c = -c if order == oracle.DESC else c
                        assert c < 0 or (c == 0 and x < y), (name, seq, order)
