"""The C-ABI library loads, exports every symbol include/gns.h declares, and
rejects bad arguments on the host before any device work (CPU only)."""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2402_01816_gb300 import build
    build.build()
    from paper_2402_01816_gb300 import _native
    return _native.lib()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            src = re.sub(r"//[^\n]*", "", src)
            names |= set(re.findall(r"\b(gns_[a-z0-9_]+)\s*\(", src))
    return names - {"gns_alloc_fn", "gns_free_fn"}


def test_exports_every_declared_symbol(L):
    declared = _declared()
    assert len(declared) >= 15
    for name in sorted(declared):
        assert hasattr(L, name), f"{name} declared in include/ but not exported"


def test_strerror_and_version(L):
    from paper_2402_01816_gb300 import _native
    for code in (0, -1, -2, -3, -4, -5):
        assert L.gns_strerror(code)
    assert b"sm_103a" in L.gns_version()
    assert _native.strerror(-5) == "device-side wait timed out"


FAKE = 1 << 40   # a device-looking address; validation fails before any use


@pytest.mark.parametrize("args,code", [
    ((FAKE, None, -1, 0, 1.0), -1),            # n < 0
    ((None, None, 10, 0, 1.0), -1),            # NULL keys with n > 0
    ((FAKE, None, 10, 2, 1.0), -1),            # unknown order
    ((FAKE, None, 10, 0, math.nan), -1),       # NaN buffer fraction
    ((FAKE, None, 10, 0, -0.5), -1),           # negative buffer fraction
    ((FAKE, None, 10, 0, 0.01), -2),           # below the smallest Frogsort2 inner fraction (1/64)
    ((FAKE + 4, None, 10, 0, 1.0), -1),        # keys not 8-byte aligned
    ((FAKE, FAKE + 2, 10, 0, 1.0), -1),        # payload misaligned
    ((FAKE, FAKE + 40, 10, 0, 1.0), -1),       # keys and payload overlap
    ((None, None, 0, 0, 1.0), 0),              # n == 0 is a no-op
    ((FAKE, None, 1, 0, 0.5), 0),              # n == 1 is a no-op
])
def test_host_argument_checks(L, args, code):
    k, p, n, order, bf = args
    for fn in (L.gns_sort, L.gns_sort_i64):
        assert fn(k, p, n, order, bf, None) == code


def test_allocator_failure_is_oom(L):
    ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
    FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
    calls = []

    @ALLOC
    def fail_alloc(nbytes, stream, ctx):
        calls.append(nbytes)
        return None

    @FREE
    def no_free(p, stream, ctx):
        raise AssertionError("free of a failed allocation")

    L.gns_set_allocator(ctypes.cast(fail_alloc, ctypes.c_void_p), ctypes.cast(no_free, ctypes.c_void_p), None)
    try:
        assert L.gns_sort(FAKE, FAKE + (1 << 30), 1 << 20, 0, 1.0, None) == -3
        assert L.gns_sort(FAKE, None, 1 << 20, 1, 0.5, None) == -3
        assert len(calls) == 2 and calls[0] >= 12 * (1 << 20)
    finally:
        L.gns_set_allocator(None, None, None)


def test_workspace_bytes_match_tiers(L):
    n = 1 << 27
    full = L.gns_workspace_bytes(n, 1.0, 0)
    half = L.gns_workspace_bytes(n, 0.5, 0)
    # %RAM = (12 n + workspace) / 12 n  (Sustainability measures section)
    ram_full = (12 * n + full) / (12 * n)
    ram_half = (12 * n + half) / (12 * n)
    assert 2.0 <= ram_full < 2.01
    assert 1.5 <= ram_half < 1.51
    # Frogsort2: floor(p n) buffer slots (Frogsort2 section)
    for p in (0.25, 0.1):
        ram = (12 * n + L.gns_workspace_bytes(n, p, 0)) / (12 * n)
        assert 1 + p <= ram < 1 + p + 0.01, (p, ram)
    assert L.gns_workspace_bytes(1, 1.0, 0) == 0
    assert L.gns_workspace_bytes(4096, 1.0, 0) <= 4096


def test_segmented_host_argument_checks(L):
    # nseg < 0, bad key type, bad order, NULL offsets with segments, misaligned offsets
    assert L.gns_segmented_sort_ex(FAKE, 1, None, FAKE, -1, 10, 0, None) == -1
    assert L.gns_segmented_sort_ex(FAKE, 7, None, FAKE, 1, 10, 0, None) == -1
    assert L.gns_segmented_sort_ex(FAKE, 1, None, FAKE, 1, 10, 3, None) == -1
    assert L.gns_segmented_sort_ex(FAKE, 1, None, None, 1, 10, 0, None) == -1
    assert L.gns_segmented_sort_ex(FAKE, 1, None, FAKE + 4, 1, 10, 0, None) == -1
    assert L.gns_segmented_sort_ex(FAKE, 1, None, FAKE, 0, 0, 0, None) == 0     # nothing to sort
    assert L.gns_segmented_sort(FAKE, None, FAKE, -2, None) == -1
    assert L.gns_segmented_sort(FAKE, None, FAKE, 0, None) == 0


def test_learned_half_plan_fits_every_size(L):
    """The half-buffer learned sort's host-side memory plan (leaf scratch carved
    from the slots free at each step) fits for every n from 2^22 on: all small
    sizes near the threshold (both parities of every subtree), and random and
    power-of-two sizes up to 2^33."""
    import random
    rng = random.Random(5)
    sizes = list(range(1 << 22, (1 << 22) + 600))
    sizes += [1 << k for k in range(22, 34)] + [(1 << k) - 1 for k in range(23, 34)]
    sizes += [rng.randrange(1 << 22, 1 << 33) for _ in range(3000)]
    for n in sizes:
        assert L.gns_learned_half_plan_ok(n) == 1, n
    assert L.gns_learned_half_plan_ok((1 << 22) - 1) == 0       # below the threshold: plain sort


@pytest.mark.parametrize("n", [1 << 27, 1 << 31])
def test_learned_half_buffer_ram(L, n):
    """%RAM = (12 n + workspace) / 12 n of the half-buffer learned sort: the
    floor(n/2) + 1024 buffer slots, the merge levels' chunk records (under
    1/16 byte per key) and a fixed few tens of MiB (network, splitters,
    key-to-bucket table, plans), i.e. about 1.5."""
    from paper_2402_01816_gb300 import _native as nat
    ws = nat.gns_workspace_bytes(n, 0.5, nat.WS_LEARNED)
    assert 12 * (n // 2) <= ws <= 12 * (n // 2 + 1024) + n // 16 + (32 << 20)
    assert 1.0 + ws / (12.0 * n) < 1.52
    # a full buffer: the partition's 16 n bytes dominate
    assert nat.gns_workspace_bytes(n, 1.0, nat.WS_LEARNED) >= 16 * n


@pytest.mark.parametrize("bf", [0.5, 0.75, 0.4, 0.3, 0.25, 0.125, 0.1, 1.0 / 32, 1.0 / 64])
def test_frog_plan_invariants(L, bf):
    """The trees of the in-place tiers, built on the host by the library's own
    split (Frogsort1) and planner (Frogsort2): children split each node
    exactly, every node can hold its inner child in its buffer, the leaves
    tile the input in order, every data slot lies in the n + buffer slots,
    chunk numbering is consecutive, and (Frogsort2) the interleaved ticket
    order maps one to one onto each depth's chunks with every node's chunk
    positions in ticket order.  Sizes near tile multiples, odd sizes, and up
    to 2^31."""
    import random
    L.gns_frog_plan_check.argtypes = [ctypes.c_int64, ctypes.c_double]
    L.gns_frog_plan_check.restype = ctypes.c_int
    rng = random.Random(7)
    T = 8192
    sizes = [T + 1, 2 * T - 1, 2 * T, 2 * T + 1, 3 * T + 5, 37 * T + 11, (1 << 18) + 12345, (1 << 20) - 1]
    sizes += [rng.randrange(T + 1, 1 << 26) for _ in range(40)]
    sizes += [(1 << 27), (1 << 27) + 7, (1 << 31)] if bf >= 0.1 else [(1 << 27) + 7]
    for n in sizes:
        assert L.gns_frog_plan_check(n, bf) == 0, (n, bf)
    assert L.gns_frog_plan_check(T, bf) == -1            # one tile: no tree


@pytest.mark.parametrize("args,code", [
    ((FAKE, None, -1, 0), -1),                 # n < 0
    ((None, None, 10, 0), -1),                 # NULL keys with n > 0
    ((FAKE, None, 10, 2), -1),                 # unknown order
    ((FAKE + 4, None, 10, 0), -1),             # keys not 8-byte aligned
    ((FAKE, FAKE + 2, 10, 0), -1),             # payload misaligned
    ((FAKE, FAKE + 40, 10, 0), -1),            # keys and payload overlap
    ((FAKE + 32, FAKE, 10, 0), -1),            # payload overlapping the keys from below
    ((FAKE, None, (1 << 20) + 1, 0), -2),      # beyond the fixed scratch: use gns_sort
    ((None, None, 0, 0), 0),                   # n == 0 is a no-op
    ((FAKE, None, 1, 1), 0),                   # n == 1 is a no-op
])
def test_noalloc_host_argument_checks(L, args, code):
    """gns_sort_noalloc rejects what gns_sort rejects, and sizes beyond its
    fixed scratch, before any device work."""
    k, p, n, order = args
    assert L.gns_sort_noalloc(k, p, n, order, None) == code


@pytest.mark.parametrize("args", [
    (FAKE, None, -1, 0, 1.0), (None, None, 10, 0, 1.0), (FAKE, None, 10, 2, 1.0),
    (FAKE, None, 10, 0, math.nan), (FAKE + 4, None, 10, 0, 1.0), (FAKE, FAKE + 40, 10, 0, 1.0),
])
def test_learned_host_argument_checks(L, args):
    k, p, n, order, bf = args
    assert L.gns_learned_sort(k, p, n, order, bf, None, None, None) == -1


@pytest.mark.parametrize("args,code", [
    ((FAKE, 0, None, 10, 0, 0.5, 3), -1),                 # unknown variant
    ((FAKE, 0, None, 10, 0, 0.5, -1), -1),
    ((FAKE, 2, None, 10, 0, 0.5, 1), -1),                 # unknown key type
    ((FAKE, 0, None, -1, 0, 0.5, 1), -1),                 # n < 0
    ((None, 0, None, 10, 0, 0.5, 2), -1),                 # NULL keys with n > 0
    ((FAKE, 0, None, 10, 2, 0.5, 2), -1),                 # unknown order
    ((FAKE + 4, 0, None, 10, 0, 0.5, 1), -1),             # keys not 8-byte aligned
    ((FAKE, 1, FAKE + 40, 10, 0, 0.5, 2), -1),            # keys and payload overlap
    ((FAKE, 0, None, 10, 0, math.nan, 2), -1),            # NaN buffer fraction
    ((FAKE, 0, None, 10, 0, -0.5, 2), -1),                # negative buffer fraction
    ((FAKE, 0, None, 10, 0, 1.0, 2), -2),                 # no in-place layout at 100%
    ((FAKE, 0, None, 10, 0, 0.01, 1), -2),                # below the smallest Frogsort2 inner fraction
])
def test_symmetric_host_argument_checks(L, args, code):
    assert L.gns_sort_symmetric(*args, None) == code


def test_symmetric_trivial_sizes_are_no_ops(L):
    assert L.gns_sort_symmetric(None, 0, None, 0, 0, 0.5, 2, None) == 0
    assert L.gns_sort_symmetric(FAKE, 1, None, 1, 1, 0.25, 1, None) == 0


@pytest.mark.parametrize("args", [
    (FAKE, 0, None, 10, FAKE, 0, 0),                      # no segment
    (FAKE, 0, None, 10, None, 2, 0),                      # NULL offsets
    (FAKE, 2, None, 10, FAKE, 2, 0),                      # unknown key type
    (FAKE, 0, None, 10, FAKE, 2, 2),                      # unknown order
    (FAKE, 0, None, -1, FAKE, 2, 0),                      # n < 0
    (None, 0, None, 10, FAKE, 2, 0),                      # NULL keys with n > 0
    (FAKE + 4, 0, None, 10, FAKE, 2, 0),                  # keys not 8-byte aligned
    (FAKE, 0, FAKE + 2, 10, FAKE, 2, 0),                  # payload not 4-byte aligned
    (FAKE, 0, None, 10, FAKE + 4, 2, 0),                  # offsets not 8-byte aligned
])
def test_ordered_segments_host_argument_checks(L, args):
    assert L.gns_debug_ordered_segments(*args, None) == -1
