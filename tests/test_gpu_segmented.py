"""Parity of gns_segmented_sort with the oracle (each segment stably sorted on
its own), bit-exact, for every size-class schedule, and at the full batched
workload (65,536 log-normal segments, about 2^28 int64 keys)."""
import os

import numpy as np
import pytest

import oracle
from paper_2402_01816_gb300 import inputs
from tests.gpu_util import assert_bitexact, need_gpu, to_dev_keys, to_dev_payload, torch

pytestmark = pytest.mark.gpu

TILE = 4096


def _offsets(lengths):
    off = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(lengths, out=off[1:])
    return off


def _run(keys, off, order=0, with_payload=True, schedule=None, repeat=1):
    import paper_2402_01816_gb300 as g
    n = keys.size
    pay = inputs.index_payload(n)
    ot = torch.from_numpy(off).cuda()
    if schedule is not None:
        os.environ["GNS_SEG_SCHEDULE"] = str(schedule)
    try:
        g.gns_segmented_release()
        for _ in range(repeat):
            kt = to_dev_keys(keys)
            pt = to_dev_payload(pay) if with_payload else None
            g.gns_segmented_sort(kt, pt, ot, order=order)
            assert g.gns_stream_status() == 0
            got_k = kt.cpu().numpy()
            got_p = None if pt is None else pt.cpu().numpy().view(np.uint32)
            want_k, want_p = oracle.segmented_sort(keys, pay if with_payload else None, off,
                                                   oracle.DESC if order else oracle.ASC)
            assert_bitexact(got_k, got_p, want_k, want_p)
        if schedule is not None:
            assert g.gns_segmented_schedule(n, ot) == schedule
    finally:
        os.environ.pop("GNS_SEG_SCHEDULE", None)


LENGTH_SETS = {
    "tiny_and_empty": [0, 1, 2, 0, 3, 16, 0, 17, 31, 1, 0],
    "tile_edges": [TILE - 1, TILE, TILE + 1, 2 * TILE - 1, 2 * TILE, 2 * TILE + 1, 1023, 1024, 1025, 2047, 2048,
                   2049, 4 * TILE + 1],
    "multi_level": [5 * TILE + 7, 33 * TILE + 1, 2, (1 << 17) + 3, 100, 9 * TILE],
    "one_big": [(1 << 19) + 5],
}


@pytest.mark.parametrize("schedule", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("name", sorted(LENGTH_SETS))
def test_length_sets_int64(name, schedule):
    need_gpu()
    lengths = LENGTH_SETS[name]
    off = _offsets(lengths)
    rng = np.random.default_rng(len(name))
    keys = rng.integers(-2**63, 2**63 - 1, int(off[-1]), dtype=np.int64, endpoint=True)
    _run(keys, off, schedule=schedule)


@pytest.mark.parametrize("order", [0, 1])
def test_lognormal_ties_f64(order):
    need_gpu()
    lengths = inputs.segment_lengths(3000, seed=4, median=300.0, hi=1 << 16)
    off = _offsets(lengths)
    keys = inputs.make_keys("ties", int(off[-1]), seed=4)
    _run(keys, off, order=order)


def test_keys_only_and_replay():
    """Keys without payload; a second call on the same pointers replays the
    captured graph and must give the same exact result."""
    need_gpu()
    lengths = inputs.segment_lengths(500, seed=8, median=2000.0, hi=1 << 15)
    off = _offsets(lengths)
    keys = np.random.default_rng(8).integers(-50, 50, int(off[-1])).astype(np.int64)
    _run(keys, off, with_payload=False, repeat=1)
    _run(keys, off, with_payload=True, repeat=2)


def test_edge_keys_f64():
    need_gpu()
    alpha = inputs.edge_alphabet()
    lengths = [7, 5000, 0, 12000, 1]
    off = _offsets(lengths)
    keys = alpha[np.random.default_rng(2).integers(0, alpha.size, int(off[-1]))]
    _run(keys, off, order=0)
    _run(keys, off, order=1)


def test_full_batched_workload():
    """65,536 segments with log-normal lengths (median 2^10, clipped 16..2^20),
    int64 keys uniform over the full range: every segment sorted and stable,
    permutation inside each segment, and 24 sampled segments bit-exact against
    the oracle."""
    need_gpu()
    import paper_2402_01816_gb300 as g
    keys, pay, off = inputs.segments(65536, seed=0)
    n = keys.size
    kt, pt = to_dev_keys(keys), to_dev_payload(pay)
    ot = torch.from_numpy(off).cuda()
    g.gns_segmented_sort(kt, pt, ot)
    assert g.gns_stream_status() == 0
    k_out = kt.cpu().numpy()
    p_out = pt.cpu().numpy().view(np.uint32)
    del kt, pt
    seg_id = np.repeat(np.arange(off.size - 1), np.diff(off))
    # payload is a permutation that stays inside each segment, moving the keys
    assert np.array_equal(seg_id[p_out], seg_id)
    assert np.array_equal(np.sort(p_out), np.arange(n, dtype=np.uint32))
    assert np.array_equal(k_out, keys[p_out])
    # sorted and stable inside segments
    same = seg_id[1:] == seg_id[:-1]
    d = np.diff(k_out)
    assert np.all(d[same] >= 0)
    tie = same & (d == 0)
    assert np.all(p_out[1:][tie] > p_out[:-1][tie])
    rng = np.random.default_rng(1)
    for s in rng.integers(0, off.size - 1, 24):
        a, b = off[s], off[s + 1]
        wk, wp = oracle.stable_sort(keys[a:b], pay[a:b])
        assert np.array_equal(k_out[a:b], wk) and np.array_equal(p_out[a:b], wp)
