"""Host side of the 1e10-key window check (test helper, not a test module).

The oracle cannot build a function over 1e10 keys in test time, but level 0
of that function is fixed, window by window, by the keys hashed into each
window (Algorithm 2 decides a position from its own keys only).  These
helpers draw the key stream on the host with the shared input generator and
keep, for each window, the keys whose level-0 position falls inside it; the
work is split over processes started with `spawn` (each runs the oracle's
single-threaded selection on its own range of keys).
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def _select_range(args):
    key_seed, j0, j1, s0, m0, windows = args
    import oracle
    from paper_1702_03154_gb300 import inputs
    parts = [[] for _ in windows]
    chunk = 1 << 21
    for a in range(j0, j1, chunk):
        b = min(j1, a + chunk)
        k = inputs.splitmix64_keys(b - a, key_seed, start=a)
        for i, (lo, W) in enumerate(windows):
            s = oracle.select_window(k, s0, m0, lo, W)
            if s.size:
                parts[i].append(s)
    return [np.concatenate(p) if p else np.empty(0, dtype=np.uint64) for p in parts]


def start_selection(n: int, key_seed: int, s0: int, m0: int, windows, workers: int = 0):
    """Start selecting, for each (lo, W) in windows, the keys of the stream
    (outputs 0..n-1 of SplitMix64(key_seed)) whose level-0 position on m0
    positions with seed s0 lies in [lo, lo + W).  Returns (pool, async
    results); `finish_selection` collects them."""
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    step = -(-n // (4 * workers))
    jobs = [(key_seed, a, min(n, a + step), s0, m0, list(windows)) for a in range(0, n, step)]
    pool = mp.get_context("spawn").Pool(workers)
    return pool, pool.map_async(_select_range, jobs)


def finish_selection(handle, timeout: float = 1800.0):
    pool, res = handle
    try:
        parts = res.get(timeout)
    except BaseException:
        pool.terminate()  # workers that cannot start are otherwise respawned forever
        raise
    pool.close()
    pool.join()
    nwin = len(parts[0]) if parts else 0
    return [np.concatenate([p[i] for p in parts]) for i in range(nwin)]


def pack_bits(A: np.ndarray) -> np.ndarray:
    """Byte-per-bit array (length a multiple of 64) as little-endian 64-bit words."""
    return np.packbits(A.astype(np.uint8), bitorder="little").view(np.uint64)
