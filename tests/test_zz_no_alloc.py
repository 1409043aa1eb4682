"""gns_sort_noalloc: the stable sort for callers that cannot allocate.

Some callers cannot let a library allocate device memory when they need a
sort: real-time or signal-safe paths where an allocator call (which may lock,
synchronise the device or map memory) is not allowed, hosts that reserve all
device memory up front and hand a library only the buffers it works on, and
code under a fixed memory budget.  gns_sort_noalloc sorts with a fixed scratch
array built into the library instead.  These tests call it through the C ABI
and check, for several calls in a row on the same scratch (the array keeps the
previous call's contents, so no call may depend on what the one before left
there), that its output is exactly what the allocating entry point gns_sort
gives and exactly the oracle's stable sort, and that it never goes to the
allocator.

This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2402_01816_gb300 import inputs
from tests.gpu_util import need_gpu, to_dev_keys, to_dev_payload, torch

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2402_01816_gb300 import build, _native
    build.build()
    return _native.lib()


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _with_gns_sort(keys, order, with_payload):
    """The same input through the existing, allocating entry point."""
    import paper_2402_01816_gb300 as g
    kt = to_dev_keys(keys)
    pt = to_dev_payload(inputs.index_payload(keys.size)) if with_payload else None
    g.gns_sort(kt, pt, order=order, buffer_fraction=1.0)
    torch.cuda.synchronize()
    return kt.cpu().numpy(), None if pt is None else pt.cpu().numpy().view(np.uint32)


def _noalloc(L, keys, order, with_payload):
    kt = to_dev_keys(keys)
    pt = to_dev_payload(inputs.index_payload(keys.size)) if with_payload else None
    rc = L.gns_sort_noalloc(ctypes.c_void_p(kt.data_ptr()), None if pt is None else ctypes.c_void_p(pt.data_ptr()),
                            keys.size, order, _stream())
    assert rc == 0, rc
    assert L.gns_stream_status(_stream()) == 0
    return kt.cpu().numpy(), None if pt is None else pt.cpu().numpy().view(np.uint32)


# (pattern, n, order, payload): several calls in a row on the one scratch array
CASES = [
    ("uniform", 1 << 20, 0, True),          # the maximum size, ascending (7 merge levels: odd)
    ("ties", 300_001, 1, True),             # smaller, descending, ragged tail (6 levels: even)
    ("permut", 123_457, 0, False),          # keys only
    ("asc_noise", 1 << 19, 0, True),        # nearly sorted, after random inputs left the scratch dirty
    ("desc", 200_000, 0, True),             # strictly descending: the single-reversal path
    ("ascall", 65_536, 0, True),            # already sorted: detection only
    ("uniform", 5_000, 1, True),            # one tile, no merge level
    ("permut", 8_193, 0, True),             # one element past a tile
]


def test_noalloc_matches_gns_sort_and_oracle_on_calls_in_a_row():
    need_gpu()
    L = _lib()
    # a failing allocator: any allocation attempt by the library would surface
    ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
    FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
    calls = []

    @ALLOC
    def no_alloc(nbytes, stream, ctx):
        calls.append(nbytes)
        return None

    @FREE
    def no_free(p, stream, ctx):
        calls.append(-1)

    inputs_ = [inputs.make_keys(p, n, seed=21) for p, n, _, _ in CASES]
    want = [_with_gns_sort(k, o, wp) for k, (_, _, o, wp) in zip(inputs_, CASES)]
    L.gns_set_allocator(ctypes.cast(no_alloc, ctypes.c_void_p), ctypes.cast(no_free, ctypes.c_void_p), None)
    try:
        got = [_noalloc(L, k, o, wp) for k, (_, _, o, wp) in zip(inputs_, CASES)]
    finally:
        L.gns_set_allocator(None, None, None)
    assert calls == []
    for keys, (p, n, o, wp), (wk, wv), (gk, gv) in zip(inputs_, CASES, want, got):
        # the allocating entry point's result, bit for bit
        assert np.array_equal(gk.view(np.uint64), wk.view(np.uint64)), (p, n, o)
        if wp:
            assert np.array_equal(gv, wv), (p, n, o)
        # and the oracle's stable sort (ties in input order), bit for bit
        ok, ov = oracle.stable_sort(keys, inputs.index_payload(n) if wp else None, o)
        assert np.array_equal(gk.view(np.uint64), ok.view(np.uint64)), (p, n, o)
        if wp:
            assert np.array_equal(gv, ov), (p, n, o)


def test_noalloc_rejects_sizes_beyond_the_scratch():
    need_gpu()
    L = _lib()
    big = (1 << 20) + 1
    kt = torch.zeros(big, dtype=torch.float64, device="cuda")
    rc = L.gns_sort_noalloc(ctypes.c_void_p(kt.data_ptr()), None, big, 0, _stream())
    assert rc == -2          # GNS_ERR_UNSUPPORTED: use gns_sort
    assert L.gns_sort_noalloc(ctypes.c_void_p(kt.data_ptr()), None, -1, 0, _stream()) == -1
