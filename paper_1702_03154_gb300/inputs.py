"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module only draws inputs; it holds none of the MPHF's own arithmetic and
is imported by both sides of a parity test (the CUDA path's callers and the
CPU oracle's callers).

Keys.  The paper's workloads are unique pseudo-random 64-bit integers
(Sec. 4, "a key is a binary representation of a pseudo-random positive
integer", unique within a file).  Key j of stream ``seed`` is output j
(0-based) of the SplitMix64 generator started at state ``seed``:
``key(j; seed) = fin(seed + (j + 1) * 0x9E3779B97F4A7C15 mod 2^64)`` with
``fin`` the published SplitMix64 output function.  The map j -> key is a
bijection of 64-bit integers, so any range of j gives distinct keys.

Shuffled query order: a seeded permutation (numpy PCG64).
Set / request sizes: log-uniform integers from a SplitMix64 stream.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)


def _splitmix_output(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _C1
    z ^= z >> np.uint64(27)
    z *= _C2
    z ^= z >> np.uint64(31)
    return z


def splitmix64_keys(n: int, seed: int, start: int = 0, chunk: int = 1 << 24) -> np.ndarray:
    """Distinct uint64 keys: outputs start .. start+n-1 of SplitMix64(seed)."""
    out = np.empty(int(n), dtype=np.uint64)
    s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        for lo in range(0, int(n), chunk):
            hi = min(int(n), lo + chunk)
            j = np.arange(start + lo + 1, start + hi + 1, dtype=np.uint64)
            out[lo:hi] = _splitmix_output(s + j * GOLDEN)
    return out


def uniform01(n: int, seed: int) -> np.ndarray:
    """n doubles in [0, 1) from the top 53 bits of a SplitMix64 stream."""
    z = splitmix64_keys(n, seed)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def log_uniform_sizes(count: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """count integer sizes, log-uniform on [lo, hi]."""
    u = uniform01(count, seed)
    v = np.floor(np.exp(u * (np.log(hi) - np.log(lo)) + np.log(lo)))
    return np.clip(v, lo, hi).astype(np.int64)


def shuffled(keys: np.ndarray, seed: int) -> np.ndarray:
    """keys in a uniformly shuffled order (seeded)."""
    perm = np.random.Generator(np.random.PCG64(seed)).permutation(keys.size)
    return keys[perm]


def sample_indices(n_total: int, count: int, seed: int) -> np.ndarray:
    """count indices drawn uniformly (with replacement) from [0, n_total)."""
    return np.random.Generator(np.random.PCG64(seed)).integers(0, n_total, size=count,
                                                               dtype=np.int64)


def set_offsets(sizes: np.ndarray) -> np.ndarray:
    """Prefix offsets (S + 1 entries) for concatenated key sets."""
    off = np.zeros(sizes.size + 1, dtype=np.uint64)
    np.cumsum(sizes.astype(np.uint64), out=off[1:])
    return off


def random_words(n: int, seed: int, length: int = 18, max_length: int = 0):
    """n random lower-case ASCII words as (uint8 bytes, n + 1 uint64 offsets).

    Every word has `length` characters, or (max_length > length) a length drawn
    uniformly from [length, max_length].  Words are drawn from PCG64(seed)
    and may repeat only by chance (26^18 choices at the default length).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if max_length > length:
        lens = rng.integers(length, max_length + 1, size=n, dtype=np.int64)
    else:
        lens = np.full(n, length, dtype=np.int64)
    off = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(lens.astype(np.uint64), out=off[1:])
    data = rng.integers(ord("a"), ord("z") + 1, size=int(off[-1]), dtype=np.uint8)
    return data, off
