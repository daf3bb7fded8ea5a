"""CPU oracle for the cascading-bit-array MPHF -- TEST INFRASTRUCTURE ONLY.

A ctypes wrapper around ``mphf_oracle.c``, a plain single-threaded C
statement of the BBhash construction (Algorithms 1-2), query (Algorithm 3),
rank checkpoints (Sec. 3.1) and fallback table (Sec. 3.5) of Limasset et al.,
arXiv 1702.03154.  Only the tests, the smoke check and the benchmark's CPU
baseline may import it; the CUDA library never does, and shares no code with
it.

Parity pins (what the oracle is checked against, in ``tests/test_oracle_*``):
the SplitMix64 published outputs, closed forms of the reduction and level
size, the worked example of Fig. 1, brute-force bijection on tiny inputs,
the expectations of Sec. 2.3 (placed fraction e^{-1/gamma}, size
gamma e^{1/gamma} N, Lemma 1), Table 1's bits/key, Sec. 3.4's temporary-set
sizes, Sec. 3.5's fallback count and order independence.  The choice of the
hash function itself (SplitMix64 finalizer) is a convention: the paper names
none, so parity with the paper's own hash values is unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mphf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libmphf_oracle.so")

OK, EINVAL, ENOMEM, EDUPLICATE = 0, 1, 2, 3
RANK_BLOCK = 512
MAX_LEVELS = 64
MASK64 = (1 << 64) - 1

POS_HOOK = ctypes.CFUNCTYPE(ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint32,
                            ctypes.c_uint64, ctypes.c_uint64)


def build_library(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        # MPHF_ORACLE_LIB lets the mutation tests load a copy of the oracle
        # compiled with a planted mistake.
        path = os.environ.get("MPHF_ORACLE_LIB") or build_library()
        L = ctypes.CDLL(path)
        u64, u32, dbl, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double, ctypes.c_void_p
        pu64 = ctypes.POINTER(ctypes.c_uint64)
        L.oracle_mix.argtypes, L.oracle_mix.restype = [u64], u64
        L.oracle_level_seed.argtypes, L.oracle_level_seed.restype = [u64, u32], u64
        L.oracle_hash.argtypes, L.oracle_hash.restype = [u64, u64], u64
        L.oracle_fastrange.argtypes, L.oracle_fastrange.restype = [u64, u64], u64
        L.oracle_level_bits.argtypes, L.oracle_level_bits.restype = [u64, dbl], u64
        L.oracle_build_hooked.argtypes = [vp, u64, dbl, u32, u64, POS_HOOK, vp, ctypes.POINTER(vp)]
        L.oracle_build_hooked.restype = ctypes.c_int
        L.oracle_build.argtypes = [vp, u64, dbl, u32, u64, ctypes.POINTER(vp)]
        L.oracle_build.restype = ctypes.c_int
        L.oracle_free.argtypes, L.oracle_free.restype = [vp], None
        L.oracle_lookup.argtypes, L.oracle_lookup.restype = [vp, vp, u64, vp], None
        L.oracle_query.argtypes, L.oracle_query.restype = [vp, u64], u64
        L.oracle_key_level.argtypes, L.oracle_key_level.restype = [vp, u64], u32
        L.oracle_num_levels.argtypes, L.oracle_num_levels.restype = [vp], u32
        L.oracle_total_bits.argtypes, L.oracle_total_bits.restype = [vp], u64
        L.oracle_num_fallback.argtypes, L.oracle_num_fallback.restype = [vp], u64
        L.oracle_num_rank.argtypes, L.oracle_num_rank.restype = [vp], u64
        L.oracle_level_info.argtypes = [vp, u32, pu64, pu64, pu64, pu64]
        L.oracle_level_info.restype = ctypes.c_int
        L.oracle_copy_bits.argtypes, L.oracle_copy_bits.restype = [vp, vp], None
        L.oracle_copy_collision_bits.argtypes = [vp, u32, vp]
        L.oracle_copy_collision_bits.restype = ctypes.c_int
        L.oracle_copy_rank.argtypes, L.oracle_copy_rank.restype = [vp, vp], None
        L.oracle_copy_fallback.argtypes, L.oracle_copy_fallback.restype = [vp, vp], None
        L.oracle_bits_per_key.argtypes, L.oracle_bits_per_key.restype = [vp], dbl
        L.oracle_bits_per_key_sampled.argtypes = [vp, u64]
        L.oracle_bits_per_key_sampled.restype = dbl
        L.oracle_string_key.argtypes, L.oracle_string_key.restype = [vp, u64, u64], u64
        L.oracle_fill_level.argtypes, L.oracle_fill_level.restype = [vp, u64, u64, u64, vp, vp], None
        L.oracle_merge_fill.argtypes, L.oracle_merge_fill.restype = [vp, vp, vp, vp, u64], None
        L.oracle_select_window.argtypes = [vp, u64, u64, u64, u64, u64, vp]
        L.oracle_select_window.restype = u64
        L.oracle_fill_window.argtypes = [vp, u64, u64, u64, u64, u64, vp, vp]
        L.oracle_fill_window.restype = None
        L.oracle_window_ranks.argtypes = [vp, u64, u64, u64, u64, u64, vp, vp]
        L.oracle_window_ranks.restype = ctypes.c_int
        L.oracle_string_keys.argtypes, L.oracle_string_keys.restype = [vp, vp, u64, u64, vp], None
        L.oracle_part_of.argtypes, L.oracle_part_of.restype = [u64, u32, u64], u32
        L.oracle_parts.argtypes, L.oracle_parts.restype = [vp, u64, u32, u64, vp], None
        _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def mix(z: int) -> int:
    return lib().oracle_mix(z)


def level_seed(seed: int, d: int) -> int:
    return lib().oracle_level_seed(seed, d)


def fastrange(h: int, m: int) -> int:
    return lib().oracle_fastrange(h, m)


def level_bits(n: int, gamma: float) -> int:
    return lib().oracle_level_bits(n, gamma)


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__({EINVAL: "invalid argument", ENOMEM: "out of memory",
                          EDUPLICATE: "duplicate keys"}.get(code, f"error {code}"))
        self.code = code


class OracleMPHF:
    """One oracle-built function; owns the C object."""

    def __init__(self, keys, gamma: float = 2.0, levels: int = 25, seed: int = 0,
                 pos_hook=None):
        keys = np.ascontiguousarray(np.asarray(keys, dtype=np.uint64))
        self._keys_ref = keys
        h = ctypes.c_void_p()
        L = lib()
        if pos_hook is None:
            rc = L.oracle_build(_ptr(keys) if keys.size else None, keys.size, float(gamma),
                                int(levels), int(seed), ctypes.byref(h))
        else:
            def _cb(user, level, key, m):
                return int(pos_hook(int(level), int(key), int(m)))
            self._cb = POS_HOOK(_cb)
            rc = L.oracle_build_hooked(_ptr(keys) if keys.size else None, keys.size,
                                       float(gamma), int(levels), int(seed), self._cb, None,
                                       ctypes.byref(h))
        if rc != OK:
            raise OracleError(rc)
        self._h = h
        self.N = int(keys.size)
        self.gamma = float(gamma)
        self.levels_budget = int(levels)
        self.seed = int(seed)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().oracle_free(h)
            self._h = None

    # -- queries -------------------------------------------------------
    def lookup(self, keys) -> np.ndarray:
        keys = np.ascontiguousarray(np.asarray(keys, dtype=np.uint64))
        out = np.empty(keys.size, dtype=np.uint64)
        if keys.size:
            lib().oracle_lookup(self._h, _ptr(keys), keys.size, _ptr(out))
        return out

    def key_level(self, x: int) -> int:
        return lib().oracle_key_level(self._h, int(x))

    # -- structure -----------------------------------------------------
    @property
    def num_levels(self) -> int:
        return lib().oracle_num_levels(self._h)

    @property
    def total_bits(self) -> int:
        return lib().oracle_total_bits(self._h)

    @property
    def num_fallback(self) -> int:
        return lib().oracle_num_fallback(self._h)

    def level_info(self, d: int):
        """(n_d, m_d, off_d, s_d) of level d."""
        a, b, c, s = (ctypes.c_uint64() for _ in range(4))
        rc = lib().oracle_level_info(self._h, d, ctypes.byref(a), ctypes.byref(b),
                                     ctypes.byref(c), ctypes.byref(s))
        if rc != OK:
            raise OracleError(rc)
        return a.value, b.value, c.value, s.value

    def levels(self):
        return [self.level_info(d) for d in range(self.num_levels)]

    def level_sizes(self):
        """[n_0, ..., n_last, n_fb]."""
        return [self.level_info(d)[0] for d in range(self.num_levels)] + [self.num_fallback]

    def bits(self) -> np.ndarray:
        out = np.empty(self.total_bits // 64, dtype=np.uint64)
        if out.size:
            lib().oracle_copy_bits(self._h, _ptr(out))
        return out

    def level_bits_words(self, d: int) -> np.ndarray:
        n, m, off, _ = self.level_info(d)
        return self.bits()[off // 64:(off + m) // 64]

    def collision_bits(self, d: int) -> np.ndarray:
        n, m, off, _ = self.level_info(d)
        out = np.empty(m // 64, dtype=np.uint64)
        rc = lib().oracle_copy_collision_bits(self._h, d, _ptr(out))
        if rc != OK:
            raise OracleError(rc)
        return out

    def rank(self) -> np.ndarray:
        out = np.empty(lib().oracle_num_rank(self._h), dtype=np.uint64)
        if out.size:
            lib().oracle_copy_rank(self._h, _ptr(out))
        return out

    def fallback(self) -> np.ndarray:
        out = np.empty(self.num_fallback, dtype=np.uint64)
        if out.size:
            lib().oracle_copy_fallback(self._h, _ptr(out))
        return out

    def bits_per_key(self) -> float:
        return lib().oracle_bits_per_key(self._h)

    def bits_per_key_sampled(self, rank_block: int) -> float:
        """Size with one 64-bit rank counter every rank_block bits (1024: minirank)."""
        return lib().oracle_bits_per_key_sampled(self._h, rank_block)


def fill_level(keys, s_d: int, m: int):
    """ArrayFill of one level over `keys`: byte arrays (A, C) of m positions."""
    k = np.ascontiguousarray(keys, dtype=np.uint64)
    A = np.zeros(m, dtype=np.uint8)
    C = np.zeros(m, dtype=np.uint8)
    lib().oracle_fill_level(_ptr(k) if k.size else None, k.size, s_d & MASK64, m, _ptr(A), _ptr(C))
    return A, C


def select_window(keys, s_d: int, m: int, lo: int, W: int) -> np.ndarray:
    """The keys (input order) whose position on a level of m positions with
    seed s_d lies in [lo, lo + W)."""
    k = np.ascontiguousarray(keys, dtype=np.uint64)
    out = np.empty(max(1, k.size), dtype=np.uint64)
    c = lib().oracle_select_window(_ptr(k) if k.size else None, k.size, s_d & MASK64, m, lo, W,
                                   _ptr(out)) if k.size else 0
    return out[:c].copy()


def fill_window(keys, s_d: int, m: int, lo: int, W: int):
    """ArrayFill of one level of m positions restricted to [lo, lo + W):
    byte arrays (A, C) of W entries; keys hashed elsewhere are skipped."""
    k = np.ascontiguousarray(keys, dtype=np.uint64)
    A = np.zeros(W, dtype=np.uint8)
    C = np.zeros(W, dtype=np.uint8)
    if k.size:
        lib().oracle_fill_window(_ptr(k), k.size, s_d & MASK64, m, lo, W, _ptr(A), _ptr(C))
    return A, C


def window_ranks(keys, s_d: int, m: int, lo: int, A) -> np.ndarray:
    """Per key: ones of the window bits A (position lo + t at entry t) before
    the key's position, if that position is in the window with its bit set;
    else UINT64_MAX."""
    k = np.ascontiguousarray(keys, dtype=np.uint64)
    a = np.ascontiguousarray(A, dtype=np.uint8)
    out = np.empty(k.size, dtype=np.uint64)
    if k.size:
        rc = lib().oracle_window_ranks(_ptr(k), k.size, s_d & MASK64, m, lo, a.size, _ptr(a),
                                       _ptr(out))
        if rc != OK:
            raise OracleError(rc)
    return out


def merge_fill(A1, C1, A2, C2):
    """Fill of the union of two disjoint key sets from their two fills (new arrays)."""
    A = np.array(A1, dtype=np.uint8, copy=True)
    C = np.array(C1, dtype=np.uint8, copy=True)
    a2 = np.ascontiguousarray(A2, dtype=np.uint8)
    c2 = np.ascontiguousarray(C2, dtype=np.uint8)
    lib().oracle_merge_fill(_ptr(A), _ptr(C), _ptr(a2), _ptr(c2), A.size)
    return A, C


def string_key(s: bytes, seed: int = 0) -> int:
    """64-bit key of one byte string (the library's string convention)."""
    buf = ctypes.create_string_buffer(bytes(s), max(1, len(s)))
    return lib().oracle_string_key(buf, len(s), seed & MASK64)


def string_keys(data: np.ndarray, offsets: np.ndarray, seed: int = 0) -> np.ndarray:
    """Keys of the strings data[offsets[i]:offsets[i+1]] (uint8 data, n+1 offsets)."""
    data = np.ascontiguousarray(data, dtype=np.uint8)
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    n = off.size - 1
    out = np.empty(n, dtype=np.uint64)
    if n:
        lib().oracle_string_keys(_ptr(data) if data.size else None, _ptr(off), n, seed & MASK64,
                                 _ptr(out))
    return out


def part_of(x: int, K: int, part_seed: int) -> int:
    """The part of K that key x belongs to."""
    return lib().oracle_part_of(int(x) & MASK64, int(K), int(part_seed) & MASK64)


def parts(keys, K: int, part_seed: int) -> np.ndarray:
    """Part of every key (uint32 array)."""
    k = np.ascontiguousarray(keys, dtype=np.uint64)
    out = np.empty(k.size, dtype=np.uint32)
    if k.size:
        lib().oracle_parts(_ptr(k), k.size, int(K), int(part_seed) & MASK64, _ptr(out))
    return out


class PartitionedOracle:
    """K independent functions, one per part of the keys (each built by the
    oracle over its part's keys, in input order); a key's global index is
    the size of the parts before its own plus its index within its part."""

    def __init__(self, keys, K: int, part_seed: int, gamma: float = 2.0, levels: int = 25,
                 seed: int = 0):
        keys = np.ascontiguousarray(np.asarray(keys, dtype=np.uint64))
        self.K, self.part_seed = int(K), int(part_seed)
        p = parts(keys, K, part_seed)
        self.functions = [OracleMPHF(keys[p == k], gamma=gamma, levels=levels, seed=seed)
                          for k in range(self.K)]
        sizes = np.array([f.N for f in self.functions], dtype=np.uint64)
        self.offsets = np.zeros(self.K + 1, dtype=np.uint64)
        np.cumsum(sizes, out=self.offsets[1:])
        self.N = int(self.offsets[-1])

    def lookup(self, q) -> np.ndarray:
        q = np.ascontiguousarray(np.asarray(q, dtype=np.uint64))
        p = parts(q, self.K, self.part_seed)
        out = np.full(q.size, MASK64, dtype=np.uint64)
        for k in range(self.K):
            sel = p == k
            if not sel.any():
                continue
            loc = self.functions[k].lookup(q[sel])
            hit = loc != np.uint64(MASK64)
            loc[hit] += self.offsets[k]
            out[sel] = loc
        return out


def build(keys, gamma: float = 2.0, levels: int = 25, seed: int = 0, pos_hook=None) -> OracleMPHF:
    return OracleMPHF(keys, gamma=gamma, levels=levels, seed=seed, pos_hook=pos_hook)


if __name__ == "__main__":  # pragma: no cover
    build_library(force="--force" in sys.argv)
    print(_LIB)
