"""Parity of gns_sort (both memory tiers) with the oracle's definition of the
stable sort, element by element and bit-exact (keys and payload)."""
import numpy as np
import pytest

import oracle
from paper_2402_01816_gb300 import inputs
from tests.gpu_util import assert_bitexact, from_dev, need_gpu, to_dev_keys, to_dev_payload, torch

pytestmark = pytest.mark.gpu

TILE = 4096      # sizes around 4096 and 8192: the tile edges of the tile sorts (8192) and of the
                 # segmented sort's big class (4096), and the merge chunks (2048)
SIZES = [0, 1, 2, 3, 17, 255, TILE - 1, TILE, TILE + 1, 2 * TILE - 1, 2 * TILE, 2 * TILE + 1, 3 * TILE + 5,
         4 * TILE + 1, 5 * TILE, 7 * TILE + 3, 16 * TILE, 16 * TILE + 1, 33 * TILE + 77, (1 << 18) + 12345]
TIERS = [1.0, 0.5]


def _run(keys, order, bf, with_payload=True):
    import paper_2402_01816_gb300 as g
    n = keys.size
    pay = inputs.index_payload(n)
    kt = to_dev_keys(keys)
    pt = to_dev_payload(pay) if with_payload else None
    g.gns_sort(kt, pt, order=order, buffer_fraction=bf)
    assert g.gns_stream_status() == 0
    got_k, got_p = from_dev(kt, pt)
    want_k, want_p = oracle.stable_sort(keys, pay if with_payload else None,
                                        oracle.DESC if order == 1 else oracle.ASC)
    assert_bitexact(got_k, got_p, want_k, want_p)


@pytest.mark.parametrize("bf", TIERS)
@pytest.mark.parametrize("n", SIZES)
def test_uniform_sizes(n, bf):
    need_gpu()
    _run(inputs.make_keys("uniform", n, seed=n), 0, bf)


@pytest.mark.parametrize("bf", TIERS)
@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("pattern", ["permut", "ties", "asc_noise", "desc", "tielog2", "asclocal",
                                     "ascglobal", "desclocal", "descglobal", "ascall", "descall",
                                     "presorted_runs", "mixture"])
def test_patterns(pattern, order, bf):
    need_gpu()
    n = 70 * TILE + 1234
    _run(inputs.make_keys(pattern, n, seed=3), order, bf)


@pytest.mark.parametrize("bf", TIERS)
@pytest.mark.parametrize("order", [0, 1])
def test_edge_keys_and_int64(order, bf):
    need_gpu()
    rng = np.random.default_rng(7)
    alpha = inputs.edge_alphabet()
    for n in (5, TILE + 3, 9 * TILE + 1):
        _run(alpha[rng.integers(0, alpha.size, n)], order, bf)
        _run(rng.integers(-2**63, 2**63 - 1, n, dtype=np.int64, endpoint=True), order, bf)
        _run(rng.integers(-3, 3, n).astype(np.int64), order, bf)


@pytest.mark.parametrize("bf", TIERS)
def test_all_equal_and_two_values(bf):
    need_gpu()
    for n in (TILE * 3 + 7, 100000):
        _run(np.full(n, 2.5), 0, bf)
        _run(np.full(n, 2.5), 1, bf)
        k = np.where(np.arange(n) % 3 == 0, 1.0, -1.0)
        _run(k, 0, bf)


@pytest.mark.parametrize("bf", TIERS)
def test_keys_only(bf):
    need_gpu()
    for n in (3, TILE + 1, 20 * TILE + 9):
        _run(inputs.make_keys("ties", n, seed=1), 0, bf, with_payload=False)


@pytest.mark.parametrize("bf", TIERS)
def test_offset_views(bf):
    """Tensors that are views at odd element offsets into a larger allocation."""
    need_gpu()
    import paper_2402_01816_gb300 as g
    n = 12 * TILE + 5
    keys = inputs.make_keys("uniform", n, seed=9)
    pay = inputs.index_payload(n)
    big_k = torch.zeros(n + 3, dtype=torch.float64, device="cuda")
    big_p = torch.zeros(n + 5, dtype=torch.int32, device="cuda")
    kt, pt = big_k[3:], big_p[1:n + 1]
    kt.copy_(torch.from_numpy(keys))
    pt.copy_(torch.from_numpy(pay.view(np.int32)))
    g.gns_sort(kt, pt, buffer_fraction=bf)
    want_k, want_p = oracle.stable_sort(keys, pay)
    got_k, got_p = from_dev(kt, pt)
    assert_bitexact(got_k, got_p, want_k, want_p)
    assert big_k[:3].abs().sum().item() == 0 and big_p[0].item() == 0 and big_p[n + 1:].abs().sum().item() == 0


def test_host_entry_point():
    need_gpu()
    import paper_2402_01816_gb300 as g
    for bf in TIERS:
        for n in (1000, 9 * TILE + 2):
            keys = inputs.make_keys("ties", n, seed=4)
            pay = inputs.index_payload(n)
            k, p = keys.copy(), pay.copy()
            g.gns_sort_host(k, p, buffer_fraction=bf)
            want_k, want_p = oracle.stable_sort(keys, pay)
            assert_bitexact(k, p, want_k, want_p)


def test_bounded_wait_timeout_then_recovery():
    """A CTA of the in-place tier skips publishing its "inputs loaded" flag: the
    CTA that depends on it gives up after the wait limit, the call reports
    GNS_ERR_TIMEOUT through the status word, and the next call is correct."""
    need_gpu()
    import paper_2402_01816_gb300 as g
    n = 1 << 16
    keys = inputs.make_keys("uniform", n, seed=12)
    kt = to_dev_keys(keys)
    g.gns_set_wait_limit_ns(20_000_000)
    try:
        g.gns_debug_skip_publish(0)
        g.gns_sort(kt, None, buffer_fraction=0.5)
        assert g.gns_stream_status() == g.GNS_ERR_TIMEOUT
        assert g.gns_stream_status() == 0       # cleared by the read
    finally:
        g.gns_debug_skip_publish(-1)
        g.gns_set_wait_limit_ns(2_000_000_000)
    _run(keys, 0, 0.5)


def test_workspace_matches_tier_ram():
    need_gpu()
    import paper_2402_01816_gb300 as g
    n = 1 << 22
    assert g.gns_workspace_bytes(n, 1.0) >= 12 * n
    assert 6 * n <= g.gns_workspace_bytes(n, 0.5) < 6.1 * n


FROG2_P = [0.25, 0.1, 0.4, 1.0 / 64]


@pytest.mark.parametrize("p", FROG2_P)
@pytest.mark.parametrize("n", [2 * TILE + 1, 5 * TILE + 3, 37 * TILE + 11, (1 << 18) + 12345])
def test_frogsort2_sizes(n, p):
    """Frogsort2 tier (buffer_fraction < 1/2): bit-exact stable sort."""
    need_gpu()
    _run(inputs.make_keys("ties", n, seed=n), 0, p)


@pytest.mark.parametrize("p", [0.25, 0.1])
@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("pattern", ["permut", "asc_noise", "tielog2", "descglobal", "mixture"])
def test_frogsort2_patterns(pattern, order, p):
    need_gpu()
    _run(inputs.make_keys(pattern, 70 * TILE + 1234, seed=5), order, p)


def test_frogsort2_workspace_is_p_of_data():
    need_gpu()
    import paper_2402_01816_gb300 as g
    n = 1 << 22
    for p in (0.25, 0.1):
        ws = g.gns_workspace_bytes(n, p)
        assert 12 * p * n <= ws < 12 * p * n + 0.12 * n    # %RAM = 1 + p + under 1% (0.12 n of 12 n bytes)


@pytest.mark.parametrize("bf", TIERS)
@pytest.mark.parametrize("n", [8, 16, 4 * TILE, 4 * TILE + 4, 8 * TILE + 2, 1 << 20])
def test_strictly_descending_sizes(n, bf):
    """Strictly descending input is reversed once (Octosort): the 16-byte
    group path (n a multiple of 8) and the element path."""
    need_gpu()
    keys = np.arange(n, 0, -1, dtype=np.float64) * 0.5
    _run(keys, 0, bf)
    _run(keys, 0, bf, with_payload=False)


@pytest.mark.parametrize("bf", [0.5, 0.25])
@pytest.mark.parametrize("order", [0, 1])
def test_presorted_nodes_skip_moves(order, bf):
    """Sorted input in the call's order with its last two keys swapped: the
    whole-array check finds no order, but every node off the rightmost path is
    presorted, so the in-place tiers leave most chunks where they are (empty
    items); the result is still exactly the stable sort."""
    need_gpu()
    n = 300 * TILE + 77
    keys = np.arange(n, dtype=np.float64)
    if order == 1:
        keys = keys[::-1].copy()
    keys[[-1, -2]] = keys[[-2, -1]]
    _run(keys, order, bf)
