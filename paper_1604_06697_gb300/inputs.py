"""Seeded synthetic inputs shaped like the paper's workloads (host, numpy).

This module holds only input generation; it contains none of the sorting
method's arithmetic.  Tests, the benchmark and the serving demo draw their
inputs here, and both the CUDA path and the CPU oracle consume the same arrays.

Generator: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), used counter-style.
For a (seed, stream) pair the state is ``s = seed ^ (stream << 32)`` and the
i-th 64-bit output is ``mix64(s + (i + 1) * 0x9E3779B97F4A7C15)``, i.e. exactly
the i-th output of a SplitMix64 generator seeded with ``s``.

Distributions follow the inputs of the paper's experiments (Sec. 4 and
Appendix A): random values, sorted, reversed, random values modulo
floor(sqrt(n)) (many duplicates), constant, and a sorted array with 1 % of its
positions swapped at random (the k-random-swaps family).
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 23

DISTRIBUTIONS = ("uniform", "sorted", "reversed", "mod_sqrt", "all_equal", "swapped_1pct")
# The structured, duplicate-heavy inputs of the paper's further experiments (Sec. 4 and
# Appendix A): A[i] = i mod floor(sqrt(n)); i^2 + n/2 mod n; i^8 + n/2 mod n; sorted
# with k random swaps of neighbouring elements (k = sqrt(n), k = n); zeros then ones;
# random zeros and ones.
EXTRA_DISTRIBUTIONS = ("i_mod_sqrt", "i2_half_mod", "i8_half_mod", "adj_swaps_sqrt", "adj_swaps_n",
                       "half_01", "random_01")
DTYPES = ("int32", "int64", "float64")


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, n: int, stream: int = 0, start: int = 0) -> np.ndarray:
    """Outputs start .. start+n-1 of the SplitMix64 stream for (seed, stream)."""
    s = np.uint64((seed ^ (stream << 32)) & 0xFFFFFFFFFFFFFFFF)
    out = np.empty(n, dtype=np.uint64)
    for c0 in range(0, n, _CHUNK):
        c1 = min(n, c0 + _CHUNK)
        idx = np.arange(start + c0 + 1, start + c1 + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            out[c0:c1] = _mix64(s + idx * GAMMA)
    return out


def unit_double(r: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of each output."""
    return (r >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def make_keys(n: int, dtype: str = "int32", dist: str = "uniform", seed: int = 0) -> np.ndarray:
    """One array of ``n`` keys of ``dtype`` drawn from distribution ``dist``."""
    if dtype not in DTYPES:
        raise ValueError(f"dtype must be one of {DTYPES}")
    npd = np.dtype(dtype)
    if dist == "uniform":
        out = np.empty(n, dtype=npd)
        for c0 in range(0, n, _CHUNK):
            c1 = min(n, c0 + _CHUNK)
            r = splitmix64(seed, c1 - c0, start=c0)
            if dtype == "int32":
                out[c0:c1] = (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.int32)
            elif dtype == "int64":
                out[c0:c1] = r.view(np.int64)
            else:
                out[c0:c1] = 2.0 * unit_double(r) - 1.0
        return out
    if dist == "sorted":
        return np.arange(n, dtype=np.int64).astype(npd)
    if dist == "reversed":
        return (n - 1 - np.arange(n, dtype=np.int64)).astype(npd)
    if dist == "mod_sqrt":
        m = max(1, math.isqrt(n))
        out = np.empty(n, dtype=npd)
        for c0 in range(0, n, _CHUNK):
            c1 = min(n, c0 + _CHUNK)
            out[c0:c1] = (splitmix64(seed, c1 - c0, start=c0) % np.uint64(m)).astype(npd)
        return out
    if dist == "all_equal":
        return np.full(n, 42, dtype=npd)
    if dist == "swapped_1pct":
        a = np.arange(n, dtype=np.int64)
        k = n // 100
        if k and n > 1:
            r = splitmix64(seed, 2 * k, stream=1) % np.uint64(n)
            u = r[0::2].astype(np.int64).tolist()
            v = r[1::2].astype(np.int64).tolist()
            for x, y in zip(u, v):   # sequential swaps, in draw order
                a[x], a[y] = a[y], a[x]
        return a.astype(npd)
    if dist in EXTRA_DISTRIBUTIONS:
        return _make_structured(n, npd, dist, seed)
    raise ValueError(f"dist must be one of {DISTRIBUTIONS + EXTRA_DISTRIBUTIONS}")


def _power_half_mod(n: int, e: int) -> np.ndarray:
    """A[i] = i^e + n/2 mod n, by repeated squaring mod n (n <= 2^32)."""
    out = np.empty(n, dtype=np.int64)
    nn = np.uint64(max(n, 1))
    for c0 in range(0, n, _CHUNK):
        c1 = min(n, c0 + _CHUNK)
        x = np.arange(c0, c1, dtype=np.uint64) % nn
        p = np.ones_like(x)
        b, k = x, e
        while k:
            if k & 1:
                p = (p * b) % nn
            b = (b * b) % nn
            k >>= 1
        out[c0:c1] = ((p + np.uint64(n // 2)) % nn).astype(np.int64)
    return out


def _make_structured(n: int, npd, dist: str, seed: int) -> np.ndarray:
    if dist == "i_mod_sqrt":
        return (np.arange(n, dtype=np.int64) % max(1, math.isqrt(n))).astype(npd)
    if dist == "i2_half_mod":
        return _power_half_mod(n, 2).astype(npd)
    if dist == "i8_half_mod":
        return _power_half_mod(n, 8).astype(npd)
    if dist in ("adj_swaps_sqrt", "adj_swaps_n"):
        a = np.arange(n, dtype=np.int64)
        k = math.isqrt(n) if dist == "adj_swaps_sqrt" else n
        if n > 1 and k:
            pos = (splitmix64(seed, k, stream=2) % np.uint64(n - 1)).astype(np.int64).tolist()
            lst = a.tolist()
            for j in pos:            # swaps of neighbours, in draw order
                lst[j], lst[j + 1] = lst[j + 1], lst[j]
            a = np.array(lst, dtype=np.int64)
        return a.astype(npd)
    if dist == "half_01":
        return (np.arange(n, dtype=np.int64) >= n // 2).astype(npd)
    # random_01
    out = np.empty(n, dtype=npd)
    for c0 in range(0, n, _CHUNK):
        c1 = min(n, c0 + _CHUNK)
        out[c0:c1] = (splitmix64(seed, c1 - c0, start=c0) >> np.uint64(63)).astype(npd)
    return out


def make_pairs(n: int, seed: int = 1, key_range: int = 1 << 20):
    """int64 keys uniform over [0, key_range) and uint32 payloads equal to the index."""
    keys = np.empty(n, dtype=np.int64)
    for c0 in range(0, n, _CHUNK):
        c1 = min(n, c0 + _CHUNK)
        keys[c0:c1] = (splitmix64(seed, c1 - c0, start=c0) % np.uint64(key_range)).astype(np.int64)
    vals = np.arange(n, dtype=np.uint32)
    return keys, vals


def segment_lengths(nseg: int, seed: int = 2, lo: int = 16, hi: int = 65536) -> np.ndarray:
    """Log-uniform lengths floor(exp(U(ln lo, ln hi))) drawn from stream 1."""
    u = unit_double(splitmix64(seed, nseg, stream=1))
    lens = np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)
    return np.clip(lens, lo, hi)


def make_segments(nseg: int, seed: int = 2, lo: int = 16, hi: int = 65536, dtype: str = "int32"):
    """``nseg`` arrays with log-uniform lengths in [lo, hi], uniform values (stream 0).

    Returns (keys, seg_offsets) with seg_offsets of length nseg + 1.
    """
    lens = segment_lengths(nseg, seed, lo, hi)
    off = np.zeros(nseg + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    keys = make_keys(int(off[-1]), dtype, "uniform", seed)
    return keys, off


def request_stream(count: int, rate_hz: float, seed: int = 3, log2_lo: float = 10.0,
                   log2_hi: float = 26.0):
    """A Poisson stream of sort requests: (arrival_s, size, dtype) per request.

    Sizes floor(2^U(log2_lo, log2_hi)), dtypes uniform over int32/int64/float64,
    exponential inter-arrival gaps of mean 1/rate_hz.
    """
    gaps = -np.log1p(-unit_double(splitmix64(seed, count, stream=1))) / rate_hz
    arrivals = np.cumsum(gaps)
    sizes = np.floor(2.0 ** (log2_lo + unit_double(splitmix64(seed, count, stream=2))
                             * (log2_hi - log2_lo))).astype(np.int64)
    dt_idx = (splitmix64(seed, count, stream=3) % np.uint64(3)).astype(np.int64)
    return [(float(a), int(s), DTYPES[d]) for a, s, d in zip(arrivals, sizes, dt_idx)]


def request_keys(index: int, size: int, dtype: str, seed: int = 3) -> np.ndarray:
    """Uniform random keys of one request (stream 16 + index of ``seed``)."""
    r = splitmix64(seed, size, stream=16 + index)
    if dtype == "int32":
        return (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.int32)
    if dtype == "int64":
        return r.view(np.int64)
    return 2.0 * unit_double(r) - 1.0
