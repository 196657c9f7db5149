"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no MergeShuffle arithmetic: it only generates the arrays and sizes of the
paper's workloads (synthetic permutations of n = 10^5..10^8 in Section 4, and the record, batched
and serving shapes this project measures). Randomness comes from splitmix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), written from its
published definition: the state advances by the golden-gamma increment and each output is the
state passed through the two xor-shift-multiply rounds of the finaliser.
"""
from __future__ import annotations

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream ids of the generators (fixed; recorded in the design notes)
S_SIZE = 0x51
S_VAL = 0x52
S_ARR = 0x53


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def splitmix64(state: np.ndarray, k: int = 1) -> np.ndarray:
    """k-th output of splitmix64 generators whose states are `state` (uint64 array)."""
    s = np.asarray(state, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(s + GOLDEN_GAMMA * np.uint64(k))


def u01(stream: int, idx: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1): top 53 bits of splitmix64(stream * 2^32 + idx)."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = splitmix64(np.uint64(stream) * np.uint64(1 << 32) + idx)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def identity_u32(n: int) -> np.ndarray:
    return np.arange(n, dtype=np.uint32)


def records16(n: int, start: int = 0, chunk: int = 1 << 24) -> np.ndarray:
    """n 16-byte records {u32 key = index, 12-byte payload} as an (n, 4) uint32 array.

    Payload bytes 0..7 are the first splitmix64 output of state `index`, bytes 8..11 the low
    32 bits of its second output."""
    out = np.empty((n, 4), dtype=np.uint32)
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        idx = np.arange(start + lo, start + hi, dtype=np.uint64)
        a = splitmix64(idx, 1)
        b = splitmix64(idx, 2)
        out[lo:hi, 0] = idx.astype(np.uint32)
        out[lo:hi, 1] = (a & np.uint64(0xFFFFFFFF)).astype(np.uint32)
        out[lo:hi, 2] = (a >> np.uint64(32)).astype(np.uint32)
        out[lo:hi, 3] = (b & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    return out


def values_u64(n: int, array_id: int = 0) -> np.ndarray:
    """Uniform 64-bit values: splitmix64(S_VAL * 2^40 + array_id * 2^27 + j)."""
    j = np.arange(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        base = np.uint64(S_VAL) * np.uint64(1 << 40) + np.uint64(array_id) * np.uint64(1 << 27)
        return splitmix64(base + j)


def batch_sizes_log_uniform(k: int, lo_log2: float, hi_log2: float, stream: int = S_SIZE
                            ) -> np.ndarray:
    """k sizes floor(2^(lo + (hi - lo) * u)) with u = u01(stream, i)."""
    u = u01(stream, np.arange(k))
    return np.floor(2.0 ** (lo_log2 + (hi_log2 - lo_log2) * u)).astype(np.uint64)


def batch_sizes_uniform(k: int, lo: int, hi: int, stream: int = S_SIZE) -> np.ndarray:
    """k sizes uniform in [lo, hi], powers of two redrawn from the next index of the stream."""
    sizes = []
    j = 0
    while len(sizes) < k:
        v = int(lo + np.floor(u01(stream, np.array([j]))[0] * (hi - lo + 1)))
        j += 1
        if v & (v - 1) == 0:
            continue
        sizes.append(v)
    return np.array(sizes, dtype=np.uint64)


def poisson_arrivals(rate_hz: float, duration_s: float, stream: int = S_ARR) -> np.ndarray:
    """Arrival times of a Poisson process: exponential gaps -ln(1 - u) / rate."""
    expected = int(rate_hz * duration_s * 1.2) + 16
    u = u01(stream, np.arange(expected))
    t = np.cumsum(-np.log1p(-u) / rate_hz)
    return t[t < duration_s]


def values_u64_torch(n: int, array_id: int = 0, device="cuda"):
    """values_u64 computed on the device with torch int64 arithmetic (same bits)."""
    import torch

    def shr(x, k):  # logical right shift of int64 bit patterns
        return (x >> k) & ((1 << (64 - k)) - 1)

    def s64(v):  # uint64 constant as a two's-complement int64
        return v - (1 << 64) if v >= (1 << 63) else v

    base = (S_VAL << 40) + (array_id << 27)
    j = torch.arange(n, dtype=torch.int64, device=device)
    z = j + s64((base + 0x9E3779B97F4A7C15) % (1 << 64))
    z = (z ^ shr(z, 30)) * s64(0xBF58476D1CE4E5B9)
    z = (z ^ shr(z, 27)) * s64(0x94D049BB133111EB)
    return z ^ shr(z, 31)
