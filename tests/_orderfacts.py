"""An independent statement of the key order, built from Python's own float and
int comparisons plus the IEEE 754 totalOrder facts for signed zeros and NaNs.
Used to pin the oracle's comparator; it shares no code with the oracle."""
import math
import struct


def bits_to_float(b: int) -> float:
    return struct.unpack("<d", struct.pack("<Q", b & (2**64 - 1)))[0]


def float_to_bits(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def f64_cmp(a_bits: int, b_bits: int) -> int:
    x, y = bits_to_float(a_bits), bits_to_float(b_bits)
    if not math.isnan(x) and not math.isnan(y):
        if x < y:
            return -1
        if x > y:
            return 1
        # numerically equal: only +0.0 / -0.0 can differ; -0.0 sorts first
        sx, sy = math.copysign(1.0, x), math.copysign(1.0, y)
        return (sx > sy) - (sx < sy)
    # NaNs: a positive-signed NaN is above everything without a NaN, a
    # negative-signed NaN below; among NaNs of one sign the payload decides
    # (larger payload = further from zero)
    def rank(bits, v):
        neg = bool(bits >> 63)
        if math.isnan(v):
            payload = bits & ((1 << 52) - 1) | ((bits >> 51) & 1) << 52
            return (-1, -payload) if neg else (1, payload)
        return (0, 0)
    ra, rb = rank(a_bits, x), rank(b_bits, y)
    if ra[0] != rb[0]:
        return -1 if ra[0] < rb[0] else 1
    if ra[0] == 0:
        raise AssertionError("unreachable")
    return (ra[1] > rb[1]) - (ra[1] < rb[1])


def i64_cmp(a: int, b: int) -> int:
    def s(v):
        v &= 2**64 - 1
        return v - 2**64 if v >= 2**63 else v
    x, y = s(a), s(b)
    return (x > y) - (x < y)
