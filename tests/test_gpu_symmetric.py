"""Parity of gns_sort_symmetric -- Frogsort1's layout in the symmetric merging
variants Geckosort1 (one branch left-ascending, the other right-ascending:
every merge reads its inner run from the far end) and Squidsort1 (the data
decides each run's orientation) -- with the oracle's stable sort, element by
element and bit-exact (keys and payload).  Whatever orientation a node's run
is stored in, the result is the unique stable sort."""
import numpy as np
import pytest

import oracle
from paper_2402_01816_gb300 import inputs
from tests.gpu_util import assert_bitexact, from_dev, need_gpu, to_dev_keys, to_dev_payload, torch

pytestmark = pytest.mark.gpu

TILE = 4096
SIZES = [0, 1, 2, 3, 255, 2 * TILE - 1, 2 * TILE, 2 * TILE + 1, 3 * TILE + 5, 4 * TILE + 1, 7 * TILE + 3,
         16 * TILE, 16 * TILE + 1, 33 * TILE + 77, (1 << 18) + 12345]
VARIANTS = {"gecko": 1, "squid": 2, "frog": 0}


def _run(keys, order, variant, with_payload=True, bf=0.5):
    import paper_2402_01816_gb300 as g
    n = keys.size
    pay = inputs.index_payload(n)
    kt = to_dev_keys(keys)
    pt = to_dev_payload(pay) if with_payload else None
    g.gns_sort_symmetric(kt, pt, order=order, variant=variant, buffer_fraction=bf)
    assert g.gns_stream_status() == 0
    got_k, got_p = from_dev(kt, pt)
    want_k, want_p = oracle.stable_sort(keys, pay if with_payload else None,
                                        oracle.DESC if order == 1 else oracle.ASC)
    assert_bitexact(got_k, got_p, want_k, want_p)


@pytest.mark.parametrize("variant", ["gecko", "squid"])
@pytest.mark.parametrize("n", SIZES)
def test_uniform_sizes(n, variant):
    need_gpu()
    _run(inputs.make_keys("uniform", n, seed=n + 1), n % 2, VARIANTS[variant])


@pytest.mark.parametrize("variant", ["gecko", "squid", "frog"])
@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("pattern", ["permut", "ties", "asc_noise", "desc", "tielog2", "asclocal", "ascglobal",
                                     "desclocal", "descglobal", "ascall", "descall", "presorted_runs", "mixture",
                                     "desc_ties", "desc_runs", "desc_noise"])
def test_patterns(pattern, order, variant):
    need_gpu()
    n = 70 * TILE + 1234
    _run(inputs.make_keys(pattern, n, seed=5), order, VARIANTS[variant])


@pytest.mark.parametrize("variant", ["gecko", "squid"])
@pytest.mark.parametrize("order", [0, 1])
def test_edge_keys_int64_and_keys_only(order, variant):
    need_gpu()
    rng = np.random.default_rng(11)
    alpha = inputs.edge_alphabet()
    v = VARIANTS[variant]
    for n in (5, TILE + 3, 9 * TILE + 1):
        _run(alpha[rng.integers(0, alpha.size, n)], order, v)
        _run(rng.integers(-2**63, 2**63 - 1, n, dtype=np.int64, endpoint=True), order, v)
        _run(rng.integers(-3, 3, n).astype(np.int64), order, v)
        _run(inputs.make_keys("ties", n, seed=2), order, v, with_payload=False)


@pytest.mark.parametrize("variant", ["gecko", "squid"])
def test_all_equal_and_mirrored_runs(variant):
    """All-equal input, and strictly descending or tied descending pieces that
    make leaves mirrored next to ascending ones (nodes whose children
    disagree read the inner run from its far end)."""
    need_gpu()
    v = VARIANTS[variant]
    n = 40 * TILE + 13
    _run(np.full(n, -1.5), 0, v)
    _run(np.full(n, -1.5), 1, v)
    i = np.arange(n)
    saw = np.where((i // (3 * TILE)) % 2 == 0, -i, i).astype(np.float64)      # alternate desc / asc runs
    _run(saw, 0, v)
    _run(saw, 1, v)
    tied = ((n - i) // 3).astype(np.float64)
    tied[n // 2:] = np.sort(tied[n // 2:])                                    # desc with ties, then asc
    _run(tied, 0, v)
    _run(tied, 1, v)


@pytest.mark.parametrize("variant", ["gecko", "squid"])
@pytest.mark.parametrize("pattern", ["permut", "desc_ties", "desc_noise"])
def test_many_levels(pattern, variant):
    """2^22 + 12345 keys: ten in-place levels, every depth of the tree."""
    need_gpu()
    n = (1 << 22) + 12345
    _run(inputs.make_keys(pattern, n, seed=7), 0, VARIANTS[variant])


def test_matches_gns_sort_half_tier():
    """GNS_FROGSORT1 through gns_sort_symmetric is gns_sort's [0.5, 1) tier."""
    need_gpu()
    import paper_2402_01816_gb300 as g
    n = 50 * TILE + 3
    keys = inputs.make_keys("asc_noise", n, seed=8)
    a, b = to_dev_keys(keys), to_dev_keys(keys)
    pa, pb = to_dev_payload(inputs.index_payload(n)), to_dev_payload(inputs.index_payload(n))
    g.gns_sort(a, pa, order=1, buffer_fraction=0.5)
    g.gns_sort_symmetric(b, pb, order=1, variant=g.FROGSORT1)
    assert torch.equal(a.view(torch.int64), b.view(torch.int64)) and torch.equal(pa, pb)


def test_offset_views():
    need_gpu()
    import paper_2402_01816_gb300 as g
    n = 12 * TILE + 5
    keys = inputs.make_keys("desc_ties", n, seed=9)
    pay = inputs.index_payload(n)
    big_k = torch.zeros(n + 3, dtype=torch.float64, device="cuda")
    big_p = torch.zeros(n + 5, dtype=torch.int32, device="cuda")
    kt, pt = big_k[3:], big_p[1:n + 1]
    kt.copy_(torch.from_numpy(keys))
    pt.copy_(torch.from_numpy(pay.view(np.int32)))
    g.gns_sort_symmetric(kt, pt, variant=g.SQUIDSORT1)
    want_k, want_p = oracle.stable_sort(keys, pay)
    got_k, got_p = from_dev(kt, pt)
    assert_bitexact(got_k, got_p, want_k, want_p)
    assert big_k[:3].abs().sum().item() == 0 and big_p[0].item() == 0 and big_p[n + 1:].abs().sum().item() == 0


@pytest.mark.parametrize("bf", [0.4, 0.25, 0.1])
@pytest.mark.parametrize("variant", ["gecko", "squid"])
@pytest.mark.parametrize("pattern", ["permut", "ties", "asc_noise", "desc_ties", "desc_runs", "descall", "uniform"])
def test_frogsort2_tree(pattern, variant, bf):
    """Geckosort and Squidsort on Frogsort2's imbalanced tree (Squidsort2 in the
    paper's table): node lists planned on the host, orientations set per call."""
    need_gpu()
    n = 70 * TILE + 1234
    order = 1 if pattern == "ties" else 0
    _run(inputs.make_keys(pattern, n, seed=13), order, VARIANTS[variant], bf=bf)


@pytest.mark.parametrize("variant", ["gecko", "squid"])
def test_frogsort2_tree_sizes_and_edges(variant):
    need_gpu()
    rng = np.random.default_rng(29)
    v = VARIANTS[variant]
    for n in (2 * TILE + 1, 5 * TILE + 3, 33 * TILE + 77, (1 << 20) + 12345):
        _run(inputs.make_keys("desc_noise", n, seed=n), n % 2, v, bf=0.25)
    alpha = inputs.edge_alphabet()
    _run(alpha[rng.integers(0, alpha.size, 9 * TILE + 1)], 1, v, bf=0.2)
    _run(rng.integers(-2**63, 2**63 - 1, 9 * TILE + 1, dtype=np.int64, endpoint=True), 0, v, bf=0.2, with_payload=False)
