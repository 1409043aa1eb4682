"""CPU oracle for the stable mergesort hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The product
library under ``paper_2402_01816_gb300/`` never imports it, and this package
imports nothing from there: the two share no code.  The only module both sides
use is the seeded input generator ``paper_2402_01816_gb300.inputs``, which holds
no sorting arithmetic.

The oracle itself is plain C (``gns_oracle.c``), compiled with gcc into
``oracle/_build/liboracle.so`` and called through ctypes on numpy arrays:

* ``stable_sort``   -- the definition of the result (Definition of sorting
                       chapter): sort (key, input index) pairs with qsort.
* ``knuthsort``     -- the paper's prior-art reference mergesort (Forgotten art
                       section: Nocopy alternation + Knuth's merge).
* ``frogsort``      -- symmetric merging with <= 50% buffer (Symmetric merging,
                       Frogsort0 and Frogsort1 sections).
* ``frog_trace``    -- slot labels after each merge level, for the layout tables
                       of the Frogsort0 / Frogsort1 sections.
* ``frogsort2``     -- Frogsort2 section: imbalanced split with inner fraction p
                       and floor(p n) buffer.
* ``omitsort`` / ``octosort`` -- Full adaptivity section: merges omitted where
                       the halves do not overlap; data-driven orientation with
                       one final reversal (100% buffer).
* ``geckosort`` / ``squidsort`` -- Symmetric merging and Squidsort sections:
                       Frogsort1's layout with mirrored orientation per branch,
                       or with the orientation decided by the data.
* ``segmented_sort``, ``final_position``, ``compare``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gns_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

F64, I64 = 0, 1
ASC, DESC = 0, 1

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2, no target-specific flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # GNS_ORACLE_LIB: load another build of gns_oracle.c (used by the
            # mutation test, which plants mistakes in copies of the source)
            path = os.environ.get("GNS_ORACLE_LIB") or build()
            lib = ctypes.CDLL(path)
            P = ctypes.c_void_p
            i64, i32 = ctypes.c_int64, ctypes.c_int
            lib.orc_compare.argtypes = [ctypes.c_uint64, ctypes.c_uint64, i32]
            lib.orc_compare.restype = i32
            lib.orc_stable_sort.argtypes = [P, P, i64, i32, i32]
            lib.orc_stable_sort.restype = i32
            lib.orc_final_position.argtypes = [P, i64, i32, i32, i64]
            lib.orc_final_position.restype = i64
            lib.orc_segmented_sort.argtypes = [P, P, P, i64, i32, i32]
            lib.orc_segmented_sort.restype = i32
            lib.orc_knuthsort.argtypes = [P, P, i64, i32, i32, P]
            lib.orc_knuthsort.restype = i32
            lib.orc_frogsort.argtypes = [P, P, i64, i32, i32, i32, P]
            lib.orc_frogsort.restype = i32
            lib.orc_frog_buffer.argtypes = [i64]
            lib.orc_frogsort2.argtypes = [P, P, i64, i32, i32, i64, i64, i64, P]
            lib.orc_frogsort2.restype = i32
            lib.orc_frog2_buffer.argtypes = [i64, i64, i64]
            lib.orc_frog2_buffer.restype = i64
            lib.orc_frog_buffer.restype = i64
            lib.orc_frog_depth.argtypes = [i64, i32]
            lib.orc_frog_depth.restype = i32
            lib.orc_frog_trace.argtypes = [i64, i32, P, i32]
            lib.orc_frog_trace.restype = i32
            lib.orc_omitsort.argtypes = [P, P, i64, i32, i32, i32, P]
            lib.orc_omitsort.restype = i32
            lib.orc_symsort.argtypes = [P, P, i64, i32, i32, i32, P]
            lib.orc_symsort.restype = i32
            _lib = lib
    return _lib


def _key_type(keys: np.ndarray) -> int:
    if keys.dtype == np.float64:
        return F64
    if keys.dtype == np.int64:
        return I64
    raise TypeError(f"oracle keys must be float64 or int64, got {keys.dtype}")


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _prep(keys, payload):
    keys = np.ascontiguousarray(keys).copy()
    if payload is not None:
        payload = np.ascontiguousarray(payload, dtype=np.uint32).copy()
        assert payload.shape == keys.shape
    return keys, payload


def compare(a_bits: int, b_bits: int, key_type: int) -> int:
    """Ascending total order of two raw 64-bit key patterns (-1, 0, +1)."""
    return _load().orc_compare(a_bits & (2**64 - 1), b_bits & (2**64 - 1), key_type)


def stable_sort(keys: np.ndarray, payload: np.ndarray | None = None, order: int = ASC):
    """The definition of the result: returns sorted copies (keys, payload)."""
    keys, payload = _prep(keys, payload)
    rc = _load().orc_stable_sort(_ptr(keys), _ptr(payload), keys.size, _key_type(keys), order)
    if rc:
        raise MemoryError("oracle stable_sort: allocation failed")
    return keys, payload


def knuthsort(keys: np.ndarray, payload: np.ndarray | None = None, order: int = ASC,
              return_counters: bool = False):
    """Paper's Knuthsort; optional counters (moves, comparisons)."""
    keys, payload = _prep(keys, payload)
    ctr = np.zeros(2, dtype=np.int64)
    rc = _load().orc_knuthsort(_ptr(keys), _ptr(payload), keys.size, _key_type(keys), order, _ptr(ctr))
    if rc:
        raise MemoryError("oracle knuthsort: allocation failed")
    if return_counters:
        return keys, payload, {"moves": int(ctr[0]), "compares": int(ctr[1])}
    return keys, payload


def frogsort(keys: np.ndarray, payload: np.ndarray | None = None, order: int = ASC,
             split_unit: int = 1, return_counters: bool = False):
    """Paper's Frogsort1 (split_unit=1) or Frogsort0 (split_unit=2, even n)."""
    keys, payload = _prep(keys, payload)
    ctr = np.zeros(3, dtype=np.int64)
    rc = _load().orc_frogsort(_ptr(keys), _ptr(payload), keys.size, _key_type(keys), order,
                              split_unit, _ptr(ctr))
    if rc == -2:
        raise ValueError("Frogsort0 needs an even number of elements")
    if rc:
        raise MemoryError("oracle frogsort: allocation failed")
    if return_counters:
        return keys, payload, {"setup_moves": int(ctr[0]), "merge_moves": int(ctr[1]),
                               "merge_compares": int(ctr[2])}
    return keys, payload


def frogsort2(keys: np.ndarray, payload: np.ndarray | None = None, order: int = ASC, p_num: int = 1,
              p_den: int = 4, leaf: int = 1, return_counters: bool = False):
    """Paper's Frogsort2 with inner fraction p = p_num / p_den (<= 1/2), using
    floor(p n) buffer slots; nodes of at most `leaf` elements are the base case."""
    keys, payload = _prep(keys, payload)
    ctr = np.zeros(3, dtype=np.int64)
    rc = _load().orc_frogsort2(_ptr(keys), _ptr(payload), keys.size, _key_type(keys), order, p_num, p_den, leaf,
                               _ptr(ctr))
    if rc == -2:
        raise ValueError("Frogsort2 needs 0 < p <= 1/2 and leaf >= 1")
    if rc == -3:
        raise AssertionError("Frogsort2 layout broke buffer >= inner child")
    if rc:
        raise MemoryError("oracle frogsort2: allocation failed")
    if return_counters:
        return keys, payload, {"setup_moves": int(ctr[0]), "merge_moves": int(ctr[1]),
                               "merge_compares": int(ctr[2])}
    return keys, payload


def _omit(keys, payload, order, lazy, return_counters):
    keys, payload = _prep(keys, payload)
    ctr = np.zeros(2, dtype=np.int64)
    rc = _load().orc_omitsort(_ptr(keys), _ptr(payload), keys.size, _key_type(keys), order, lazy, _ptr(ctr))
    if rc:
        raise MemoryError("oracle omitsort: allocation failed")
    if return_counters:
        return keys, payload, {"moves": int(ctr[0]), "compares": int(ctr[1])}
    return keys, payload


def omitsort(keys: np.ndarray, payload: np.ndarray | None = None, order: int = ASC,
             return_counters: bool = False):
    """Paper's Omitsort: merges of non-overlapping halves omitted, data location
    returned by the recursion; counters (moves, comparisons)."""
    return _omit(keys, payload, order, 0, return_counters)


def octosort(keys: np.ndarray, payload: np.ndarray | None = None, order: int = ASC,
             return_counters: bool = False):
    """Paper's Octosort: Omitsort with data-driven orientation, the target
    order enforced only where children disagree, one final reversal."""
    return _omit(keys, payload, order, 1, return_counters)


def _sym(keys, payload, order, lazy, return_counters):
    keys, payload = _prep(keys, payload)
    ctr = np.zeros(3, dtype=np.int64)
    rc = _load().orc_symsort(_ptr(keys), _ptr(payload), keys.size, _key_type(keys), order, lazy, _ptr(ctr))
    if rc:
        raise MemoryError("oracle symmetric sort: allocation failed")
    if return_counters:
        return keys, payload, {"setup_moves": int(ctr[0]), "merge_moves": int(ctr[1]),
                               "compares": int(ctr[2])}
    return keys, payload


def geckosort(keys: np.ndarray, payload: np.ndarray | None = None, order: int = ASC,
              return_counters: bool = False):
    """Paper's Geckosort (Frogsort1's layout, data-left nodes left-ascending,
    data-right nodes right-ascending); counters (setup moves, merge moves,
    comparisons)."""
    return _sym(keys, payload, order, 0, return_counters)


def squidsort(keys: np.ndarray, payload: np.ndarray | None = None, order: int = ASC,
              return_counters: bool = False):
    """Paper's Squidsort1 (Frogsort1 with Octosort's data-driven orientation and
    a non-overlap test per node)."""
    return _sym(keys, payload, order, 1, return_counters)


def frog2_buffer(n: int, p_num: int, p_den: int) -> int:
    return int(_load().orc_frog2_buffer(n, p_num, p_den))


def frog_buffer(n: int) -> int:
    return int(_load().orc_frog_buffer(n))


def frog_depth(n: int, split_unit: int = 1) -> int:
    return int(_load().orc_frog_depth(n, split_unit))


def frog_trace(n: int, split_unit: int = 1) -> np.ndarray:
    """(rows, n + n//2) int32 slot labels: +(s+1) data set up in slot s, -(s+1) buffer."""
    d = frog_depth(n, split_unit)
    m = n + n // 2
    out = np.zeros((d + 1, m), dtype=np.int32)
    rows = _load().orc_frog_trace(n, split_unit, _ptr(out), d + 1)
    if rows < 0:
        raise ValueError("frog_trace: bad arguments")
    return out[:rows]


def segmented_sort(keys: np.ndarray, payload: np.ndarray | None, offsets: np.ndarray,
                   order: int = ASC):
    keys, payload = _prep(keys, payload)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    nseg = offsets.size - 1
    rc = _load().orc_segmented_sort(_ptr(keys), _ptr(payload), _ptr(offsets), nseg,
                                    _key_type(keys), order)
    if rc:
        raise MemoryError("oracle segmented_sort: allocation failed")
    return keys, payload


def final_position(keys: np.ndarray, i: int, order: int = ASC) -> int:
    """Output position of input element i in the stable sort (O(n) rank count)."""
    keys = np.ascontiguousarray(keys)
    return int(_load().orc_final_position(_ptr(keys), keys.size, _key_type(keys), order, i))
