"""Checks without a sanitizer (compute-sanitizer is not used here):

* race detection for the in-place tiers: with the jitter test hook every
  ticket of the in-place merge levels and every setup leaf waits a random
  bounded time before loading, so tickets load in perturbed orders; a store
  that did not wait for a load it overwrites would change the result, which
  must stay bit-exact against the oracle;
* the merge-path co-ranks of one level against their definition, computed
  here with NumPy (the rank of every left-run element in the right run);
* an allocator hook that returns NULL: the call reports GNS_ERR_OOM and the
  next call sorts correctly.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2402_01816_gb300 import inputs
from tests.gpu_util import assert_bitexact, from_dev, need_gpu, to_dev_keys, to_dev_payload, torch

pytestmark = pytest.mark.gpu

TILE = 4096
CHUNK = 2048


def _sort_and_check(keys, order, fn):
    n = keys.size
    pay = inputs.index_payload(n)
    kt, pt = to_dev_keys(keys), to_dev_payload(pay)
    fn(kt, pt)
    import paper_2402_01816_gb300 as g
    assert g.gns_stream_status() == 0
    got_k, got_p = from_dev(kt, pt)
    want_k, want_p = oracle.stable_sort(keys, pay, oracle.DESC if order else oracle.ASC)
    assert_bitexact(got_k, got_p, want_k, want_p)


@pytest.mark.parametrize("pattern", ["permut", "asc_noise", "desc_ties", "ties", "desc_runs"])
@pytest.mark.parametrize("form", ["frog1", "frog2", "gecko", "squid", "squid2"])
def test_in_place_tiers_under_jitter(form, pattern):
    need_gpu()
    import paper_2402_01816_gb300 as g
    order = 1 if pattern == "ties" else 0
    n = (1 << 20) + 12345 if pattern in ("permut", "desc_ties") else 70 * TILE + 1234

    def fn(kt, pt):
        if form == "frog1":
            g.gns_sort(kt, pt, order=order, buffer_fraction=0.5)
        elif form == "frog2":
            g.gns_sort(kt, pt, order=order, buffer_fraction=0.25)
        elif form == "squid2":
            g.gns_sort_symmetric(kt, pt, order=order, variant=g.SQUIDSORT1, buffer_fraction=0.25)
        else:
            g.gns_sort_symmetric(kt, pt, order=order, variant=g.GECKOSORT1 if form == "gecko" else g.SQUIDSORT1)
    g.gns_debug_jitter(20000)
    try:
        _sort_and_check(inputs.make_keys(pattern, n, seed=17), order, fn)
    finally:
        g.gns_debug_jitter(0)


def _coranks_by_definition(keys, w):
    """splits[b] for every 2048-output chunk b, from the definition: left-run
    element i lands at output i + #(right-run keys strictly below it)."""
    n = keys.size
    out = []
    for b in range((n + CHUNK - 1) // CHUNK):
        out0 = b * CHUNK
        ps = out0 // (2 * w) * (2 * w)
        la = min(w, n - ps)
        lb = max(0, min(w, n - ps - w))
        a = keys[ps:ps + la]
        bb = keys[ps + la:ps + la + lb]
        pos = np.arange(la) + np.searchsorted(bb, a, side="left")
        out.append(int(np.count_nonzero(pos < out0 - ps)))
    return np.array(out, dtype=np.int64)


@pytest.mark.parametrize("w", [1024, 8192, 1 << 15])
@pytest.mark.parametrize("kind", ["random", "ties", "disjoint"])
def test_merge_partition_coranks(w, kind):
    need_gpu()
    import paper_2402_01816_gb300 as g
    rng = np.random.default_rng(w + len(kind))
    n = 5 * w + 1234                       # ragged: the last pair is short, the very last run shorter still
    if kind == "random":
        keys = rng.integers(0, 1 << 62, n, dtype=np.int64)
    elif kind == "ties":
        keys = rng.integers(0, 7, n, dtype=np.int64)
    else:
        keys = np.arange(n, dtype=np.int64)[::-1].copy()      # every pair of runs fully reversed
    for s in range(0, n, w):
        keys[s:s + w] = np.sort(keys[s:s + w])
    got = g.gns_debug_merge_partition(torch.from_numpy(keys).cuda(), w).cpu().numpy()
    assert np.array_equal(got, _coranks_by_definition(keys, w))


def test_allocator_returning_null_reports_oom():
    need_gpu()
    import paper_2402_01816_gb300 as g
    L = g.lib()
    ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
    FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
    calls = []

    @ALLOC
    def null_alloc(size, stream, ctx):
        calls.append(size)
        return None

    @FREE
    def no_free(p, stream, ctx):
        calls.append(-1)

    keys = inputs.make_keys("permut", 50 * TILE, seed=3)
    kt, pt = to_dev_keys(keys), to_dev_payload(inputs.index_payload(keys.size))
    L.gns_set_allocator(ctypes.cast(null_alloc, ctypes.c_void_p), ctypes.cast(no_free, ctypes.c_void_p), None)
    try:
        for bf in (1.0, 0.5):
            with pytest.raises(g.GnsError) as ei:
                g.gns_sort(kt, pt, buffer_fraction=bf)
            assert ei.value.code == g.GNS_ERR_OOM
        with pytest.raises(g.GnsError) as ei:
            g.gns_sort_symmetric(kt, pt, variant=g.SQUIDSORT1)
        assert ei.value.code == g.GNS_ERR_OOM
    finally:
        L.gns_set_allocator(None, None, None)
    assert calls and all(c > 0 for c in calls)        # asked for memory, never freed what it did not get
    # the input is untouched and the next call (default allocator) sorts it
    assert np.array_equal(kt.cpu().numpy(), keys)
    _sort_and_check(keys, 0, lambda a, b: g.gns_sort(a, b, buffer_fraction=0.5))
