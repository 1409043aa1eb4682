"""The learned sort's bucket sort on its own (gns_debug_ordered_segments): a
stable sort of ordered segments, tile-sorted at the array's global 8192-key
tiles (a tile may hold the ends of several segments) with merge levels over
each segment's own runs.  Ordered segments make the stable sort of the whole
array the result, so every case is compared element by element and bit for
bit (keys and payload) with the oracle's stable sort of the whole array.
Layouts: empty and one-key segments, segments one key either side of a tile
boundary, segments spanning many tiles at every offset, tiles holding the
ends of thousands of segments, one segment over everything, ragged tails."""
import numpy as np
import pytest

import oracle
from paper_2402_01816_gb300 import inputs
from tests.gpu_util import assert_bitexact, from_dev, need_gpu, to_dev_keys, to_dev_payload, torch

pytestmark = pytest.mark.gpu

T = 8192


def _ordered_keys(sizes, rng, kind, order):
    """Keys whose segments are ordered under `order`: segment s holds values
    around s * 2^20 (descending order: around -s * 2^20), with ties."""
    parts = []
    for s, z in enumerate(sizes):
        base = s * (1 << 20) if order == 0 else -s * (1 << 20)
        if kind == "ties":
            v = base + rng.integers(0, 3, z)
        elif kind == "equal":
            v = np.full(z, base)
        else:
            v = base + rng.integers(0, 1 << 19, z)
        parts.append(v.astype(np.int64))
    return np.concatenate(parts) if parts else np.zeros(0, dtype=np.int64)


def _run(sizes, rng, kind="random", order=0, as_float=True, with_payload=True):
    import paper_2402_01816_gb300 as g
    keys = _ordered_keys(sizes, rng, kind, order)
    if as_float:
        keys = keys.astype(np.float64) / 3.0
    n = keys.size
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    pay = inputs.index_payload(n)
    kt = to_dev_keys(keys)
    pt = to_dev_payload(pay) if with_payload else None
    g.gns_debug_ordered_segments(kt, pt, torch.from_numpy(off).cuda(), order=order)
    assert g.gns_stream_status() == 0
    got_k, got_p = from_dev(kt, pt)
    want_k, want_p = oracle.stable_sort(keys, pay if with_payload else None, oracle.DESC if order else oracle.ASC)
    assert_bitexact(got_k, got_p, want_k, want_p)


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("kind", ["random", "ties", "equal"])
def test_boundary_sizes(kind, order):
    """Segments of sizes around the tile, in every combination of offsets."""
    need_gpu()
    rng = np.random.default_rng(3 + order)
    sizes = [0, 1, T - 1, 1, T, T + 1, 0, 2 * T - 3, 5, 3 * T + 7, T // 2, T // 2, 0, 0, 9 * T + 11, 17, 64 * T + 5]
    _run(sizes, rng, kind, order)


@pytest.mark.parametrize("order", [0, 1])
def test_many_tiny_segments(order):
    """Tiles holding the ends of thousands of segments (sizes 0 to 4)."""
    need_gpu()
    rng = np.random.default_rng(11)
    sizes = rng.integers(0, 5, 20000).tolist()
    _run(sizes, rng, "random", order)


@pytest.mark.parametrize("as_float", [True, False])
def test_learned_like_layout(as_float):
    """Three hundred segments of log-normal sizes around 8 tiles, one of 200
    tiles, a ragged tail: the bucket layout of the learned sort."""
    need_gpu()
    rng = np.random.default_rng(29)
    sizes = np.clip(rng.lognormal(np.log(8 * T), 0.5, 300), 0, 40 * T).astype(np.int64).tolist()
    sizes[150] = 200 * T + 3
    _run(sizes + [12345], rng, "random", 0, as_float=as_float)


def test_single_segment_and_keys_only():
    """One segment over everything (the plain sort through this path), and a
    keys-only call."""
    need_gpu()
    rng = np.random.default_rng(41)
    _run([37 * T + 1234], rng, "random", 0)
    _run([37 * T + 1234], rng, "ties", 1, with_payload=False)
    _run([0, 0, 5, 0], rng, "random", 0)
