"""gns_sort_noalloc: the stable sort for callers that cannot allocate.

Callers that run inside somebody else's CUDA-graph capture, on paths that must
not call an allocator, or inside a host that owns all device memory cannot let
a library allocate scratch.  gns_sort_noalloc sorts with a fixed scratch array
built into the library instead.  These tests call it through the C ABI and
check that it gives exactly what gns_sort gives, on two calls in a row (the
scratch keeps the previous call's contents, so the second call must not be
affected by the first), and that it never goes to the allocator.

This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_2402_01816_gb300 import inputs
from tests.gpu_util import need_gpu, to_dev_keys, to_dev_payload, torch

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2402_01816_gb300 import build, _native
    build.build()
    return _native.lib()


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _reference(keys, order):
    """The same input through the existing, allocating entry point."""
    import paper_2402_01816_gb300 as g
    kt = to_dev_keys(keys)
    pt = to_dev_payload(inputs.index_payload(keys.size))
    g.gns_sort(kt, pt, order=order, buffer_fraction=1.0)
    torch.cuda.synchronize()
    return kt.cpu().numpy(), pt.cpu().numpy()


def _noalloc(L, keys, order):
    kt = to_dev_keys(keys)
    pt = to_dev_payload(inputs.index_payload(keys.size))
    rc = L.gns_sort_noalloc(ctypes.c_void_p(kt.data_ptr()), ctypes.c_void_p(pt.data_ptr()), keys.size, order,
                            _stream())
    assert rc == 0, rc
    assert L.gns_stream_status(_stream()) == 0
    return kt.cpu().numpy(), pt.cpu().numpy()


def test_noalloc_matches_gns_sort_twice_in_a_row():
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

    cases = [("uniform", (1 << 20), 0),            # the maximum size, ascending
             ("ties", 300_001, 1)]                 # then smaller, descending, ragged
    want = [_reference(inputs.make_keys(p, n, seed=21), o) for p, n, o in cases]
    L.gns_set_allocator(ctypes.cast(no_alloc, ctypes.c_void_p), ctypes.cast(no_free, ctypes.c_void_p), None)
    try:
        got = [_noalloc(L, inputs.make_keys(p, n, seed=21), o) for p, n, o in cases]
    finally:
        L.gns_set_allocator(None, None, None)
    assert calls == []
    for (wk, wp), (gk, gp) in zip(want, got):
        assert np.array_equal(gk.view(np.uint64), wk.view(np.uint64))
        assert np.array_equal(gp, wp)


def test_noalloc_rejects_sizes_beyond_the_scratch():
    need_gpu()
    L = _lib()
    big = (1 << 20) + 1
    kt = torch.zeros(big, dtype=torch.float64, device="cuda")
    rc = L.gns_sort_noalloc(ctypes.c_void_p(kt.data_ptr()), None, big, 0, _stream())
    assert rc == -2          # GNS_ERR_UNSUPPORTED: use gns_sort
    assert L.gns_sort_noalloc(ctypes.c_void_p(kt.data_ptr()), None, -1, 0, _stream()) == -1
