"""Pins the oracle's total order (Definition of sorting chapter; -0.0/NaN
reading: IEEE 754 totalOrder) against Python's own comparisons."""
import numpy as np
import pytest

import oracle
from paper_2402_01816_gb300 import inputs
from tests._orderfacts import f64_cmp, float_to_bits, i64_cmp


def _bits(x):
    return int(np.float64(x).view(np.uint64))


def test_f64_matches_python_on_numbers():
    rng = np.random.default_rng(1)
    vals = np.concatenate([
        rng.standard_normal(400) * 10.0 ** rng.integers(-300, 300, 400),
        np.array([0.0, -0.0, np.inf, -np.inf, 5e-324, -5e-324, 1.0, -1.0, 2.0 ** 1023]),
        rng.integers(-5, 5, 50).astype(np.float64),
    ])
    for i in range(0, vals.size, 7):
        for j in range(vals.size):
            a, b = _bits(vals[i]), _bits(vals[j])
            assert oracle.compare(a, b, oracle.F64) == f64_cmp(a, b)


def test_signed_zero_and_nan_positions():
    neg0, pos0 = float_to_bits(-0.0), float_to_bits(0.0)
    assert oracle.compare(neg0, pos0, oracle.F64) == -1
    assert oracle.compare(pos0, neg0, oracle.F64) == 1
    pinf, ninf = float_to_bits(float("inf")), float_to_bits(float("-inf"))
    for bits in (0x7ff8000000000000, 0x7ff0000000000001, 0x7fffffffffffffff):
        assert oracle.compare(bits, pinf, oracle.F64) == 1
        assert oracle.compare(ninf, bits, oracle.F64) == -1
    for bits in (0xfff8000000000000, 0xfff0000000000002):
        assert oracle.compare(bits, ninf, oracle.F64) == -1
        assert oracle.compare(bits, pinf, oracle.F64) == -1
    # NaN payload order (totalOrder): +NaN payload 1 above payload 0, -NaN reversed
    assert oracle.compare(0x7ff8000000000001, 0x7ff8000000000000, oracle.F64) == 1
    assert oracle.compare(0xfff8000000000001, 0xfff8000000000000, oracle.F64) == -1


def test_edge_alphabet_all_pairs():
    bits = [int(b) for b in inputs.edge_alphabet().view(np.uint64)]
    for a in bits:
        for b in bits:
            assert oracle.compare(a, b, oracle.F64) == f64_cmp(a, b)
            assert oracle.compare(a, b, oracle.F64) == -oracle.compare(b, a, oracle.F64)


def test_i64_matches_python():
    rng = np.random.default_rng(2)
    vals = np.concatenate([rng.integers(-2**63, 2**63 - 1, 300, endpoint=True),
                           np.array([-2**63, -1, 0, 1, 2**63 - 1], dtype=np.int64)])
    for i in range(0, vals.size, 5):
        for j in range(vals.size):
            a, b = int(vals[i]) & (2**64 - 1), int(vals[j]) & (2**64 - 1)
            assert oracle.compare(a, b, oracle.I64) == i64_cmp(a, b)
