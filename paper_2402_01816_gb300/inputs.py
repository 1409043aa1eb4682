"""Seeded synthetic inputs for the stable mergesort (no sorting arithmetic here).

This is the only module that both the CUDA path's tests/benchmark and the CPU
oracle use.  Every generator is a pure function of (size, seed): NumPy PCG64
streams from ``SeedSequence(seed).spawn(...)``, one child stream per pattern.
Payload is always the input index (uint32), so stability is visible in the
output.

Workloads (the shapes of the paper's test patterns, Methods and measurement
section, plus the four workload families of this library):

* ``uniform``      n float64 i.i.d. uniform[0, 1)
* ``permut``       a random permutation of 1..n as float64 (distinct keys)
* ``ties``         heavy ties: j / 2**13 with j uniform in [0, 2**13)
* ``asc_noise``    1..n ascending, then n/100 random transpositions
* ``desc``         n..1 strictly descending
* ``tielog2``, ``ascall``, ``asclocal``, ``ascglobal``, ``descall``,
  ``desclocal``, ``descglobal``  -- the paper's own pattern list
* ``presorted_runs`` blocks of 2**16; block b ascending iff b % 10 == 0,
  the others random (over a permutation of 1..n)
* ``desc_ties``    non-increasing with every value twice: floor((n - 1 - i) / 2)
  (descending order with ties, which a reversal would not sort stably)
* ``desc_runs``    a random permutation of 1..n cut into runs of 2**16, each
  sorted descending (``desclocal`` with runs of a fixed length well above a
  tile)
* ``desc_noise``   n..1 descending, then n/100 random transpositions
* ``mixture``      40% exp(N(0, 2^2)); 30% Zipf(s=1.2) over 1..2**16; 30% a mix
  of 8 Gaussians (mu ~ U(-10, 10), sigma log-uniform in [0.01, 1])
* ``segments``     log-normal segment lengths (median 2**10, clipped 16..2**20)
  with int64 keys uniform over the full range
"""
from __future__ import annotations

import math

import numpy as np

PATTERNS_C1 = ("permut", "ties", "asc_noise", "desc")
PAPER_PATTERNS = ("permut", "tielog2", "ascall", "asclocal", "ascglobal",
                  "descall", "desclocal", "descglobal")

_PATTERN_IDS = {name: i for i, name in enumerate(
    ("uniform", "permut", "ties", "asc_noise", "desc", "tielog2", "ascall", "asclocal",
     "ascglobal", "descall", "desclocal", "descglobal", "presorted_runs", "mixture",
     "segments", "edge", "desc_ties", "desc_runs", "desc_noise"))}


def rng_for(pattern: str, seed: int = 0) -> np.random.Generator:
    """One independent PCG64 stream per pattern name, all from one seed."""
    children = np.random.SeedSequence(seed).spawn(len(_PATTERN_IDS))
    return np.random.default_rng(children[_PATTERN_IDS[pattern]])


def index_payload(n: int) -> np.ndarray:
    return np.arange(n, dtype=np.uint32)


def _permutation_1n(rng: np.random.Generator, n: int) -> np.ndarray:
    return (rng.permutation(n) + 1).astype(np.float64)


def make_keys(pattern: str, n: int, seed: int = 0) -> np.ndarray:
    """float64 keys of one pattern (int64 for 'segments' is separate)."""
    rng = rng_for(pattern, seed)
    if pattern == "uniform":
        return rng.random(n)
    if pattern == "permut":
        return _permutation_1n(rng, n)
    if pattern == "ties":
        return rng.integers(0, 2**13, n).astype(np.float64) / 2**13
    if pattern == "asc_noise":
        k = np.arange(1, n + 1, dtype=np.float64)
        m = n // 100
        if n >= 2 and m > 0:
            a = rng.integers(0, n, m)
            b = rng.integers(0, n, m)
            for lo in range(0, m, 1 << 20):         # sequential transpositions
                for x, y in zip(a[lo:lo + (1 << 20)].tolist(), b[lo:lo + (1 << 20)].tolist()):
                    k[x], k[y] = k[y], k[x]
        return k
    if pattern == "desc":
        return np.arange(n, 0, -1, dtype=np.float64)
    if pattern == "tielog2":
        d = max(1, int(math.log2(max(n, 2))))
        vals = rng.permutation(n)[:d] + 1 if n >= d else np.arange(1, d + 1)
        return vals[rng.integers(0, d, n)].astype(np.float64)
    if pattern == "ascall":
        return np.arange(1, n + 1, dtype=np.float64)
    if pattern == "descall":
        return np.arange(n, 0, -1, dtype=np.float64)
    if pattern in ("asclocal", "desclocal"):
        # n distinct numbers randomly put into sqrt(n) presorted sequences of length sqrt(n)
        r = max(1, int(math.isqrt(n)))
        vals = _permutation_1n(rng, n)
        out = np.empty(n, dtype=np.float64)
        for s in range(0, n, r):
            blk = np.sort(vals[s:s + r])
            out[s:s + r] = blk if pattern == "asclocal" else blk[::-1]
        return out
    if pattern in ("ascglobal", "descglobal"):
        # n distinct numbers cut into sqrt(n) quantiles of length sqrt(n), each
        # randomly permuted; quantiles in ascending (descending) order
        r = max(1, int(math.isqrt(n)))
        base = np.arange(1, n + 1, dtype=np.float64)
        if pattern == "descglobal":
            base = base[::-1].copy()
        out = np.empty(n, dtype=np.float64)
        for s in range(0, n, r):
            out[s:s + r] = rng.permutation(base[s:s + r])
        return out
    if pattern == "presorted_runs":
        k = _permutation_1n(rng, n)
        blk = 1 << 16
        for bi, s in enumerate(range(0, n, blk)):
            if bi % 10 == 0:
                k[s:s + blk] = np.sort(k[s:s + blk])
        return k
    if pattern == "desc_ties":
        return ((n - 1 - np.arange(n)) // 2).astype(np.float64)
    if pattern == "desc_runs":
        vals = _permutation_1n(rng, n)
        blk = 1 << 16
        out = np.empty(n, dtype=np.float64)
        for s in range(0, n, blk):
            out[s:s + blk] = np.sort(vals[s:s + blk])[::-1]
        return out
    if pattern == "desc_noise":
        k = np.arange(n, 0, -1, dtype=np.float64)
        m = n // 100
        if n >= 2 and m > 0:
            a = rng.integers(0, n, m)
            b = rng.integers(0, n, m)
            for x, y in zip(a.tolist(), b.tolist()):
                k[x], k[y] = k[y], k[x]
        return k
    if pattern == "mixture":
        return mixture_keys(n, seed)
    raise ValueError(f"unknown pattern {pattern!r}")


def make_keys_device(pattern: str, n: int, seed: int = 0, device="cuda"):
    """Device-side generation of the two large-run patterns (permutation-based),
    for sizes where NumPy's single-threaded shuffle takes minutes: ``permut``
    (a random permutation of 1..n as float64) and ``presorted_runs`` (the same,
    with every 10th block of 2**16 ascending), from torch's seeded generator.
    Same structure as ``make_keys``; not the same numbers."""
    import torch
    if n < 2**31:
        gen = torch.Generator(device=device)
        gen.manual_seed(int(seed) * 1_000_003 + _PATTERN_IDS[pattern])
        perm = torch.randperm(n, generator=gen, device=device)
    elif n & (n - 1) == 0:
        # torch's shuffle stops at 2**31 - 1 elements: for a power of two, a
        # seeded composition of bijections of the k-bit integers (multiply by an
        # odd constant and add, mod 2**k; xor with a right shift) permutes 0..n-1
        k = n.bit_length() - 1
        rng = rng_for(pattern, seed)
        perm = torch.arange(n, dtype=torch.int64, device=device)
        for _ in range(6):
            a = 2 * int(rng.integers(1 << 20, 1 << 30)) + 1
            b = int(rng.integers(0, n))
            perm.mul_(a).add_(b).bitwise_and_(n - 1)
            perm.bitwise_xor_(perm >> ((k + 1) // 2))
    else:
        raise ValueError("device generator: n >= 2**31 must be a power of two")
    keys = (perm + 1).to(torch.float64)
    del perm
    if pattern == "permut":
        return keys
    if pattern == "presorted_runs":
        blk = 1 << 16
        nfull = n // blk
        rows = keys[: nfull * blk].view(nfull, blk)
        sel = torch.arange(0, nfull, 10, device=device)
        rows[sel] = torch.sort(rows[sel], dim=1).values
        if nfull * blk < n and nfull % 10 == 0:
            keys[nfull * blk:] = torch.sort(keys[nfull * blk:]).values
        return keys
    raise ValueError(f"no device generator for {pattern!r}")


def mixture_keys(n: int, seed: int = 0) -> np.ndarray:
    rng = rng_for("mixture", seed)
    comp = rng.choice(3, size=n, p=[0.4, 0.3, 0.3])
    out = np.empty(n, dtype=np.float64)
    i0 = np.flatnonzero(comp == 0)
    out[i0] = np.exp(rng.normal(0.0, 2.0, i0.size))
    i1 = np.flatnonzero(comp == 1)
    support = np.arange(1, 2**16 + 1, dtype=np.float64)
    w = support ** -1.2
    w /= w.sum()
    out[i1] = rng.choice(support, size=i1.size, p=w)
    i2 = np.flatnonzero(comp == 2)
    mu = rng.uniform(-10.0, 10.0, 8)
    sigma = np.exp(rng.uniform(math.log(0.01), math.log(1.0), 8))
    g = rng.integers(0, 8, i2.size)
    out[i2] = rng.normal(mu[g], sigma[g])
    return out


def segment_lengths(nseg: int = 65536, seed: int = 0, median: float = 1024.0,
                    sigma: float = math.sqrt(2.0 * math.log(4.0)),
                    lo: int = 16, hi: int = 1 << 20) -> np.ndarray:
    """Log-normal segment lengths: round(exp(ln(median) + sigma Z)) clipped to [lo, hi]."""
    rng = rng_for("segments", seed)
    z = rng.standard_normal(nseg)
    return np.clip(np.rint(np.exp(math.log(median) + sigma * z)), lo, hi).astype(np.int64)


def segments(nseg: int = 65536, seed: int = 0, **kw):
    """(keys int64 uniform over the full range, payload, offsets int64[nseg+1])."""
    lengths = segment_lengths(nseg, seed, **kw)
    offsets = np.zeros(nseg + 1, dtype=np.int64)
    np.cumsum(lengths, out=offsets[1:])
    n = int(offsets[-1])
    rng = rng_for("segments", seed + 1_000_003)
    keys = rng.integers(-2**63, 2**63 - 1, n, dtype=np.int64, endpoint=True)
    return keys, index_payload(n), offsets


def edge_alphabet() -> np.ndarray:
    """float64 bit patterns that stress the total order: signed zeros,
    infinities, quiet and signalling NaNs of both signs with distinct payloads."""
    bits = np.array([
        0x0000000000000000,  # +0.0
        0x8000000000000000,  # -0.0
        0x7ff0000000000000,  # +inf
        0xfff0000000000000,  # -inf
        0x7ff8000000000000,  # +qNaN
        0x7ff8000000000001,  # +qNaN, payload 1
        0xfff8000000000000,  # -qNaN
        0x7ff0000000000001,  # +sNaN
        0xfff0000000000002,  # -sNaN
        0x0000000000000001,  # smallest +subnormal
        0x8000000000000001,  # smallest -subnormal
        0x3ff0000000000000,  # 1.0
        0xbff0000000000000,  # -1.0
        0x7fefffffffffffff,  # max finite
        0xffefffffffffffff,  # -max finite
    ], dtype=np.uint64)
    return bits.view(np.float64)
