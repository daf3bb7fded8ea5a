"""Thin ctypes binding of ``libmphf.so`` (C ABI in ``include/mphf.h``).

Argument marshalling only: every step of construction and lookup runs in the
library's CUDA kernels.  PyTorch supplies device memory and streams; keys are
``torch.int64`` tensors holding the 64-bit key patterns (reinterpreted as
unsigned by the library).  There is no CPU fallback: if the library cannot be
built or loaded, the first call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build_ext

OK, EINVAL, ENOMEM, EDUPLICATE, ECUDA, ETIMEOUT, EINTERNAL = range(7)
NOT_FOUND = (1 << 64) - 1
RANK_BLOCK = 512
MAX_LEVELS = 64

_lib = None


class MPHFError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        L = lib()
        msg = L.mphf_strerror(code).decode()
        if code == ECUDA:
            msg += ": " + L.mphf_last_cuda_error().decode()
        super().__init__(f"{what}: {msg}" if what else msg)
        self.code = code


def _check(rc: int, what: str):
    if rc != OK:
        raise MPHFError(rc, what)


def lib_path() -> str:
    return build_ext.LIB


def lib():
    """Load (building first if needed) the in-tree CUDA library."""
    global _lib
    if _lib is not None:
        return _lib
    if not build_ext.up_to_date():
        build_ext.build()
    if not os.path.exists(build_ext.LIB):
        raise RuntimeError(f"libmphf.so is missing at {build_ext.LIB}; the CUDA path cannot run")
    L = ctypes.CDLL(build_ext.LIB)
    vp, u64, u32, dbl, i32 = (ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double,
                              ctypes.c_int)
    pvp = ctypes.POINTER(ctypes.c_void_p)
    pu64 = ctypes.POINTER(ctypes.c_uint64)
    sig = {
        "mphf_strerror": ([i32], ctypes.c_char_p),
        "mphf_last_cuda_error": ([], ctypes.c_char_p),
        "mphf_abi_version": ([], i32),
        "mphf_build": ([vp, u64, dbl, u32, u64, vp, pvp], i32),
        "mphf_build_host": ([vp, u64, dbl, u32, u64, vp, pvp], i32),
        "mphf_lookup": ([vp, vp, u64, vp, vp], i32),
        "mphf_lookup_host": ([vp, vp, u64, vp, vp], i32),
        "mphf_build_lookup_host": ([vp, u64, dbl, u32, u64, vp, u64, vp, vp, pvp], i32),
        "mphf_bits_per_key": ([vp], dbl),
        "mphf_device_bytes": ([vp], u64),
        "mphf_free": ([vp], None),
        "mphf_num_keys": ([vp], u64),
        "mphf_num_levels": ([vp, vp], i32),
        "mphf_total_bits": ([vp], u64),
        "mphf_num_rank": ([vp], u64),
        "mphf_num_fallback": ([vp], u64),
        "mphf_level_info": ([vp, u32, pu64, pu64, pu64, pu64], i32),
        "mphf_copy_bits": ([vp, vp, u64], i32),
        "mphf_copy_rank": ([vp, vp, u64], i32),
        "mphf_copy_fallback": ([vp, vp, u64], i32),
        "mphf_keygen": ([vp, u64, u64, u64, vp], i32),
        "mphf_build_path": ([vp], i32),
        "mphf_debug_config": ([i32, dbl], i32),
        "mphf_build_batched": ([vp, vp, u32, dbl, u32, u64, vp, vp], i32),
        "mphf_build_batched_host_offsets": ([vp, vp, u32, dbl, u32, u64, vp, vp], i32),
        "mphf_autotune_batched": ([vp, vp, u32, dbl, u32, u64, vp, ctypes.POINTER(dbl)], i32),
        "mphf_batched_debug_config": ([dbl], i32),
        "mphf_debug_slabs": ([u32, u64], i32),
        "mphf_debug_lookup_wide": ([i32], i32),
        "mphf_debug_size_level": ([u64, dbl, u64, pu64, pu64, pu64], i32),
        "mphf_debug_level1_bound": ([u64, dbl, u64, pu64, pu64, pu64], i32),
        "mphf_batched_tuning": ([u32, u64, pu64, pu64, pu64], i32),
        "mphf_batched_set_tuning": ([u32, u64, u64, u64, u64], i32),
        "mphf_workspace_release": ([], None),
        "mphf_rank_table_noalloc": ([vp, u64, vp, vp, vp], i32),
        "mphf_lookup_multi": ([vp, vp, vp, vp, u32, vp], i32),
        "mphf_server_create": ([u64, u32, i32, i32, u64, pvp], i32),
        "mphf_server_destroy": ([vp], None),
        "mphf_server_submit_lookup": ([vp, vp, vp, u64, vp, pu64], i32),
        "mphf_server_submit_build": ([vp, vp, u64, dbl, u32, u64, pu64], i32),
        "mphf_server_wait": ([vp, u64, dbl, ctypes.POINTER(i32), ctypes.POINTER(dbl), pvp], i32),
        "mphf_server_stats": ([vp, pu64, pu64, pu64, pu64], i32),
        "mphf_server_loadgen": ([vp, vp, vp, vp, u32, dbl, dbl, dbl, dbl, vp, u64, dbl, vp, u64,
                                 dbl, dbl, dbl, u64, vp, u64, pu64, pu64, pu64,
                                 ctypes.POINTER(dbl)], i32),
        "mphf_string_keys": ([vp, u64, vp, u64, u64, vp, vp], i32),
        "mphf_set_layout": ([vp, u32, vp], i32),
        "mphf_sector_bytes": ([vp], u32),
        "mphf_build_nodisk": ([vp, u64, dbl, u32, u64, dbl, vp, pvp], i32),
        "mphf_build_generated": ([u64, u64, u64, dbl, u32, u64, dbl, vp, pvp], i32),
        "mphf_serialized_size": ([vp, pu64], i32),
        "mphf_serialize": ([vp, vp, u64], i32),
        "mphf_deserialize": ([vp, u64, vp, pvp], i32),
        "mphf_ceiling_random_loads": ([vp, u64, u32, u64, u64, vp, vp, vp], i32),
        "mphf_ceiling_random_atomics": ([vp, u64, i32, u64, u64, vp, vp, vp], i32),
        "mphf_ceiling_copy": ([vp, vp, u64, vp], i32),
        "mphf_route": ([vp, u64, u32, u64, vp, vp, vp, vp], i32),
        "mphf_unroute": ([vp, vp, u64, vp, vp], i32),
        "mphf_add_offset": ([vp, u64, u64, vp], i32),
        "mphf_build_partitioned": ([vp, u64, u32, u64, dbl, u32, u64, vp, pvp], i32),
        "mphf_part_lookup": ([vp, vp, u64, vp, vp], i32),
        "mphf_part_info": ([vp, ctypes.POINTER(u32), vp], i32),
        "mphf_part_function": ([vp, u32], vp),
        "mphf_part_free": ([vp], None),
        "mphf_pool_trim": ([], i32),
        "mphf_server_latency_parts": ([vp, vp, vp], i32),
        "mphf_launch_count": ([], u64),
        "mphf_profile_enable": ([i32], i32),
        "mphf_profile_report": ([ctypes.c_char_p, u64], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _stream_ptr(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) or None


def _dev_keys(keys):
    import torch
    if not isinstance(keys, torch.Tensor) or not keys.is_cuda:
        raise TypeError("keys must be a CUDA tensor (use build_host / lookup_host for host arrays)")
    if keys.dtype not in (torch.int64, getattr(torch, "uint64", torch.int64)):
        raise TypeError("keys must hold 64-bit integers")
    return keys.contiguous()


def _host_u64(a) -> np.ndarray:
    try:
        import torch
        if isinstance(a, torch.Tensor):
            a = a.detach().cpu().numpy()
    except ImportError:  # pragma: no cover
        pass
    a = np.asarray(a)
    if a.dtype != np.uint64:
        a = a.astype(np.int64, copy=False).view(np.uint64) if a.dtype == np.int64 else a.astype(np.uint64)
    return np.ascontiguousarray(a)


class MPHF:
    """A minimal perfect hash function resident in GPU memory."""

    def __init__(self, handle: ctypes.c_void_p, owner=None):
        self._h = handle
        # a function owned by another object (a part of a PartitionedMPHF)
        # keeps that object alive and is never freed here
        self._owner = owner

    # -- construction ---------------------------------------------------
    @classmethod
    def build(cls, keys, gamma: float = 2.0, levels: int = 25, seed: int = 0, stream=None) -> "MPHF":
        keys = _dev_keys(keys)
        h = ctypes.c_void_p()
        rc = lib().mphf_build(keys.data_ptr() if keys.numel() else None, keys.numel(), float(gamma),
                              int(levels), int(seed) & NOT_FOUND, _stream_ptr(stream),
                              ctypes.byref(h))
        _check(rc, "mphf_build")
        return cls(h)

    @classmethod
    def build_host(cls, keys, gamma: float = 2.0, levels: int = 25, seed: int = 0,
                   stream=None) -> "MPHF":
        a = keys if isinstance(keys, np.ndarray) and keys.dtype == np.uint64 else _host_u64(keys)
        ptr = _host_ptr(keys, a)
        h = ctypes.c_void_p()
        rc = lib().mphf_build_host(ptr if a.size else None, a.size, float(gamma), int(levels),
                                   int(seed) & NOT_FOUND, _stream_ptr(stream), ctypes.byref(h))
        _check(rc, "mphf_build_host")
        return cls(h)

    @classmethod
    def build_lookup_host(cls, keys, queries, out: Optional[np.ndarray] = None,
                          gamma: float = 2.0, levels: int = 25, seed: int = 0, stream=None):
        """Build from host keys and look up host queries in one pipelined call.

        Returns (function, indices): the same as build_host then lookup_host."""
        a = keys if isinstance(keys, np.ndarray) and keys.dtype == np.uint64 else _host_u64(keys)
        qa = (queries if isinstance(queries, np.ndarray) and queries.dtype == np.uint64
              else _host_u64(queries))
        if out is None:
            out = np.empty(qa.size, dtype=np.uint64)
        h = ctypes.c_void_p()
        rc = lib().mphf_build_lookup_host(_host_ptr(keys, a) if a.size else None, a.size,
                                          float(gamma), int(levels), int(seed) & NOT_FOUND,
                                          _host_ptr(queries, qa) if qa.size else None, qa.size,
                                          _host_ptr(out, out) if qa.size else None,
                                          _stream_ptr(stream), ctypes.byref(h))
        _check(rc, "mphf_build_lookup_host")
        return cls(h), out

    @classmethod
    def build_nodisk(cls, keys, gamma: float = 2.0, levels: int = 25, seed: int = 0,
                     keep_fraction: float = 0.02, stream=None) -> "MPHF":
        """Build without storing F_d: every level re-reads the caller's keys (Sec. 3.4)."""
        keys = _dev_keys(keys)
        h = ctypes.c_void_p()
        rc = lib().mphf_build_nodisk(keys.data_ptr() if keys.numel() else None, keys.numel(),
                                     float(gamma), int(levels), int(seed) & NOT_FOUND,
                                     float(keep_fraction), _stream_ptr(stream), ctypes.byref(h))
        _check(rc, "mphf_build_nodisk")
        return cls(h)

    @classmethod
    def build_generated(cls, n: int, key_seed: int, key_start: int = 0, gamma: float = 2.0,
                        levels: int = 25, seed: int = 0, keep_fraction: float = 0.02,
                        stream=None) -> "MPHF":
        """Build over the SplitMix64 keys key(j), j < n, generated on the fly (Sec. 4.5)."""
        h = ctypes.c_void_p()
        rc = lib().mphf_build_generated(int(n), int(key_seed) & NOT_FOUND,
                                        int(key_start) & NOT_FOUND, float(gamma), int(levels),
                                        int(seed) & NOT_FOUND, float(keep_fraction),
                                        _stream_ptr(stream), ctypes.byref(h))
        _check(rc, "mphf_build_generated")
        return cls(h)

    # -- rank sampling -------------------------------------------------------
    def set_layout(self, sector_bytes: int, stream=None) -> None:
        """Re-store A and its ranks in 32-byte sectors (default), 64-byte sectors
        ("minirank", smaller) or 8-byte units (faster lookups, larger)."""
        _check(lib().mphf_set_layout(self._h, int(sector_bytes), _stream_ptr(stream)),
               "mphf_set_layout")

    @property
    def sector_bytes(self) -> int:
        return lib().mphf_sector_bytes(self._h)

    # -- serialization -------------------------------------------------------
    def to_bytes(self) -> bytes:
        """The function as a self-contained byte image (mphf_serialize)."""
        n = ctypes.c_uint64()
        _check(lib().mphf_serialized_size(self._h, ctypes.byref(n)), "mphf_serialized_size")
        buf = np.empty(n.value, dtype=np.uint8)
        _check(lib().mphf_serialize(self._h, buf.ctypes.data, n.value), "mphf_serialize")
        return buf.tobytes()

    @classmethod
    def from_bytes(cls, image, stream=None) -> "MPHF":
        """A new function on the current device from an image made by to_bytes."""
        a = np.frombuffer(image, dtype=np.uint8)
        h = ctypes.c_void_p()
        _check(lib().mphf_deserialize(a.ctypes.data if a.size else None, a.size,
                                      _stream_ptr(stream), ctypes.byref(h)), "mphf_deserialize")
        return cls(h)

    def save(self, path: str) -> None:
        with open(path, "wb") as f:
            f.write(self.to_bytes())

    @classmethod
    def load(cls, path: str, stream=None) -> "MPHF":
        with open(path, "rb") as f:
            return cls.from_bytes(f.read(), stream)

    def free(self):
        if self._owner is None and self._h is not None and self._h.value:
            lib().mphf_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:  # pragma: no cover - interpreter shutdown
            pass

    @property
    def handle(self) -> int:
        return self._h.value

    # -- queries ----------------------------------------------------------
    def lookup(self, keys, out=None, stream=None):
        import torch
        keys = _dev_keys(keys)
        if out is None:
            out = torch.empty(keys.numel(), dtype=torch.int64, device=keys.device)
        rc = lib().mphf_lookup(self._h, keys.data_ptr(), keys.numel(), out.data_ptr(),
                               _stream_ptr(stream))
        _check(rc, "mphf_lookup")
        return out

    def lookup_host(self, keys, out: Optional[np.ndarray] = None, stream=None) -> np.ndarray:
        a = keys if isinstance(keys, np.ndarray) and keys.dtype == np.uint64 else _host_u64(keys)
        if out is None:
            out = np.empty(a.size, dtype=np.uint64)
        rc = lib().mphf_lookup_host(self._h, _host_ptr(keys, a), a.size, _host_ptr(out, out),
                                    _stream_ptr(stream))
        _check(rc, "mphf_lookup_host")
        return out

    # -- structure ----------------------------------------------------------
    def bits_per_key(self) -> float:
        return lib().mphf_bits_per_key(self._h)

    def device_bytes(self) -> int:
        """Device memory held by the function (A, rank table with in-block counts, fallback)."""
        return lib().mphf_device_bytes(self._h)

    @property
    def build_path(self) -> int:
        """1 = bucketed (shared-memory) construction, 2 = unbucketed (L2 atomics),
        3 = batched construction, 4 = loaded from a serialized image."""
        return lib().mphf_build_path(self._h)

    @property
    def N(self) -> int:
        return lib().mphf_num_keys(self._h)

    @property
    def num_levels(self) -> int:
        v = ctypes.c_uint32()
        _check(lib().mphf_num_levels(self._h, ctypes.byref(v)), "mphf_num_levels")
        return v.value

    @property
    def total_bits(self) -> int:
        return lib().mphf_total_bits(self._h)

    @property
    def num_rank(self) -> int:
        return lib().mphf_num_rank(self._h)

    @property
    def num_fallback(self) -> int:
        return lib().mphf_num_fallback(self._h)

    def level_info(self, d: int):
        a, b, c, s = (ctypes.c_uint64() for _ in range(4))
        _check(lib().mphf_level_info(self._h, d, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                     ctypes.byref(s)), "mphf_level_info")
        return a.value, b.value, c.value, s.value

    def levels(self):
        return [self.level_info(d) for d in range(self.num_levels)]

    def level_sizes(self):
        return [self.level_info(d)[0] for d in range(self.num_levels)] + [self.num_fallback]

    def bits(self) -> np.ndarray:
        out = np.empty(self.total_bits // 64, dtype=np.uint64)
        _check(lib().mphf_copy_bits(self._h, out.ctypes.data if out.size else None, out.size),
               "mphf_copy_bits")
        return out

    def rank(self) -> np.ndarray:
        out = np.empty(self.num_rank, dtype=np.uint64)
        _check(lib().mphf_copy_rank(self._h, out.ctypes.data if out.size else None, out.size),
               "mphf_copy_rank")
        return out

    def fallback(self) -> np.ndarray:
        out = np.empty(self.num_fallback, dtype=np.uint64)
        _check(lib().mphf_copy_fallback(self._h, out.ctypes.data if out.size else None, out.size),
               "mphf_copy_fallback")
        return out


def _host_ptr(orig, arr: np.ndarray) -> Optional[int]:
    """Pointer to host data; a pinned torch CPU tensor is passed through as is."""
    try:
        import torch
        if isinstance(orig, torch.Tensor) and not orig.is_cuda and orig.is_contiguous() \
                and orig.element_size() == 8:
            return orig.data_ptr() if orig.numel() else None
    except ImportError:  # pragma: no cover
        pass
    return arr.ctypes.data if arr.size else None


def _is_cuda_tensor(x) -> bool:
    try:
        import torch
        return isinstance(x, torch.Tensor) and x.is_cuda
    except ImportError:  # pragma: no cover
        return False


def _offsets(offsets) -> np.ndarray:
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.uint64))
    if off.ndim != 1 or off.size < 2:
        raise ValueError("offsets must hold S + 1 entries")
    return off


def build_batched(keys, offsets, gamma: float = 2.0, levels: int = 25, seed: int = 0,
                  stream=None) -> list:
    """One function per key set: set s is keys[offsets[s]:offsets[s+1]].

    offsets: S + 1 entries, either a CUDA tensor (int64 / uint64; passed to
    mphf_build_batched) or host integers (mphf_build_batched_host_offsets)."""
    keys = _dev_keys(keys)
    kp = keys.data_ptr() if keys.numel() else None
    if _is_cuda_tensor(offsets):
        if offsets.dim() != 1 or offsets.numel() < 2 or offsets.element_size() != 8:
            raise ValueError("offsets must hold S + 1 64-bit entries")
        off_t = offsets.contiguous()
        S = off_t.numel() - 1
        arr = (ctypes.c_void_p * S)()
        rc = lib().mphf_build_batched(kp, off_t.data_ptr(), S, float(gamma), int(levels),
                                      int(seed) & NOT_FOUND, _stream_ptr(stream), arr)
        _check(rc, "mphf_build_batched")
        return [MPHF(ctypes.c_void_p(arr[i])) for i in range(S)]
    off = _offsets(offsets)
    S = off.size - 1
    arr = (ctypes.c_void_p * S)()
    rc = lib().mphf_build_batched_host_offsets(kp, off.ctypes.data, S, float(gamma), int(levels),
                                               int(seed) & NOT_FOUND, _stream_ptr(stream), arr)
    _check(rc, "mphf_build_batched_host_offsets")
    return [MPHF(ctypes.c_void_p(arr[i])) for i in range(S)]


def autotune_batched(keys, offsets, gamma: float = 2.0, levels: int = 25, seed: int = 0,
                     stream=None) -> float:
    keys = _dev_keys(keys)
    off = _offsets(offsets)
    best = ctypes.c_double(0.0)
    rc = lib().mphf_autotune_batched(keys.data_ptr() if keys.numel() else None, off.ctypes.data,
                                     off.size - 1, float(gamma), int(levels), int(seed) & NOT_FOUND,
                                     _stream_ptr(stream), ctypes.byref(best))
    _check(rc, "mphf_autotune_batched")
    return best.value


def debug_size_level(n: int, gamma: float, btarget: int) -> tuple:
    """(B, cap, P): the bucketed level size the device picks for n keys."""
    v = [ctypes.c_uint64() for _ in range(3)]
    _check(lib().mphf_debug_size_level(int(n), float(gamma), int(btarget),
                                       *[ctypes.byref(x) for x in v]), "mphf_debug_size_level")
    return tuple(x.value for x in v)


def debug_level1_bound(N: int, gamma: float, btarget: int) -> tuple:
    """(n1_hi, capY, Bb): level 1's arena bound of a bucketed build of N keys."""
    v = [ctypes.c_uint64() for _ in range(3)]
    _check(lib().mphf_debug_level1_bound(int(N), float(gamma), int(btarget),
                                         *[ctypes.byref(x) for x in v]), "mphf_debug_level1_bound")
    return tuple(x.value for x in v)


def debug_lookup_wide(on: bool = True) -> None:
    """Test hook: every lookup through the 64-bit position kernels."""
    _check(lib().mphf_debug_lookup_wide(1 if on else 0), "mphf_debug_lookup_wide")


def debug_slabs(shift: int = 27, min_ac_bytes: int = 64 << 20) -> None:
    """Test hook: slab size and threshold of the unbucketed path's key grouping."""
    _check(lib().mphf_debug_slabs(int(shift), int(min_ac_bytes)), "mphf_debug_slabs")


def batched_tuning(S: int, total_keys: int) -> dict:
    """What mphf_autotune_batched chose for S sets of total_keys keys (None if never tuned)."""
    v = [ctypes.c_uint64() for _ in range(3)]
    rc = lib().mphf_batched_tuning(int(S), int(total_keys), *[ctypes.byref(x) for x in v])
    if rc != OK:
        return None
    return dict(zip(("bucket_width_max", "buckets_per_set_max", "tail_keys"), (x.value for x in v)))


def batched_set_tuning(S: int, total_keys: int, bucket_width_max: int,
                       buckets_per_set_max: int, tail_keys: int) -> None:
    """Pins the batched build's choice for this size class (see batched_tuning)."""
    _check(lib().mphf_batched_set_tuning(int(S), int(total_keys), int(bucket_width_max),
                                         int(buckets_per_set_max), int(tail_keys)),
           "mphf_batched_set_tuning")


def batched_debug_config(cap_scale: float = 1.0):
    _check(lib().mphf_batched_debug_config(float(cap_scale)), "mphf_batched_debug_config")


def workspace_release():
    lib().mphf_workspace_release()


def build(keys, gamma: float = 2.0, levels: int = 25, seed: int = 0, stream=None) -> MPHF:
    return MPHF.build(keys, gamma=gamma, levels=levels, seed=seed, stream=stream)


def keygen(n: int, seed: int, start: int = 0, device=None, stream=None):
    """n distinct keys on the device: outputs start.. of SplitMix64(seed)."""
    import torch
    out = torch.empty(int(n), dtype=torch.int64, device=device or "cuda")
    if n:
        _check(lib().mphf_keygen(out.data_ptr(), int(n), int(seed) & NOT_FOUND, int(start),
                                 _stream_ptr(stream)), "mphf_keygen")
    return out


def string_keys(data, offsets, seed: int = 0, stream=None):
    """64-bit keys (int64 CUDA tensor) of the byte strings data[offsets[i]:offsets[i+1]].

    data: uint8 bytes (numpy array, bytes, or a CUDA uint8 tensor); offsets:
    n + 1 non-decreasing offsets (numpy or CUDA int64/uint64 tensor).
    """
    import torch
    if isinstance(data, (bytes, bytearray)):
        data = np.frombuffer(bytes(data), dtype=np.uint8)
    if isinstance(data, np.ndarray):
        data = torch.from_numpy(np.ascontiguousarray(data, dtype=np.uint8)).cuda()
    if isinstance(offsets, np.ndarray):
        offsets = torch.from_numpy(np.ascontiguousarray(offsets, dtype=np.uint64).view(np.int64)).cuda()
    data = data.contiguous()
    offsets = offsets.contiguous()
    n = offsets.numel() - 1
    out = torch.empty(max(n, 0), dtype=torch.int64, device=offsets.device)
    if n > 0:
        rc = lib().mphf_string_keys(data.data_ptr() if data.numel() else None, data.numel(),
                                    offsets.data_ptr(), n, int(seed) & NOT_FOUND, out.data_ptr(),
                                    _stream_ptr(stream))
        _check(rc, "mphf_string_keys")
    return out


def debug_config(path: int = 0, cap_scale: float = 1.0):
    """Test hook: path 0 = bucketed with fallback (default), 1 = unbucketed only;
    cap_scale < 1 shrinks bucket capacities so that the fallback is taken."""
    _check(lib().mphf_debug_config(int(path), float(cap_scale)), "mphf_debug_config")


def lookup_multi(handles, keys_list, outs_list=None, stream=None):
    """One launch answering several lookup requests against different functions."""
    import torch
    n = len(handles)
    keys_list = [_dev_keys(k) for k in keys_list]
    if outs_list is None:
        outs_list = [torch.empty(k.numel(), dtype=torch.int64, device=k.device) for k in keys_list]
    H = (ctypes.c_void_p * n)(*[h.handle for h in handles])
    K = (ctypes.c_void_p * n)(*[k.data_ptr() for k in keys_list])
    O = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs_list])
    C = (ctypes.c_uint64 * n)(*[k.numel() for k in keys_list])
    _check(lib().mphf_lookup_multi(H, K, O, C, n, _stream_ptr(stream)), "mphf_lookup_multi")
    return outs_list


class Server:
    """The C serving loop (continuous batching of lookups, admitted builds)."""

    def __init__(self, max_batch_keys=1 << 22, max_batch_reqs=4096, max_inflight=3,
                 build_workers=1, mem_reserve=2 << 30):
        p = ctypes.c_void_p()
        _check(lib().mphf_server_create(int(max_batch_keys), int(max_batch_reqs),
                                        int(max_inflight), int(build_workers), int(mem_reserve),
                                        ctypes.byref(p)), "mphf_server_create")
        self._p = p
        self._keep = {}

    def close(self):
        if self._p is not None and self._p.value:
            lib().mphf_server_destroy(self._p)
        self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # pragma: no cover
            pass

    def submit_lookup(self, h: "MPHF", keys, out) -> int:
        rid = ctypes.c_uint64()
        _check(lib().mphf_server_submit_lookup(self._p, h.handle, keys.data_ptr(), keys.numel(),
                                               out.data_ptr(), ctypes.byref(rid)),
               "mphf_server_submit_lookup")
        self._keep[rid.value] = (keys, out)
        return rid.value

    def submit_build(self, keys, gamma=2.0, levels=25, seed=0) -> int:
        rid = ctypes.c_uint64()
        _check(lib().mphf_server_submit_build(self._p, keys.data_ptr(), keys.numel(), float(gamma),
                                              int(levels), int(seed) & NOT_FOUND,
                                              ctypes.byref(rid)), "mphf_server_submit_build")
        self._keep[rid.value] = (keys,)
        return rid.value

    def wait(self, rid: int, timeout: float = 600.0):
        """(status, latency_s, built MPHF or None)."""
        st, lat, built = ctypes.c_int(), ctypes.c_double(), ctypes.c_void_p()
        rc = lib().mphf_server_wait(self._p, rid, float(timeout), ctypes.byref(st),
                                    ctypes.byref(lat), ctypes.byref(built))
        if rc != OK:
            raise MPHFError(rc, "mphf_server_wait")
        self._keep.pop(rid, None)
        return st.value, lat.value, (MPHF(built) if built.value else None)

    def stats(self):
        v = [ctypes.c_uint64() for _ in range(4)]
        _check(lib().mphf_server_stats(self._p, *[ctypes.byref(x) for x in v]), "mphf_server_stats")
        return dict(zip(("batches", "requests", "keys", "builds"), (x.value for x in v)))

    def loadgen(self, handles, keys_list, rate_hz, duration_s, bmin, bmax, out, build_frac=0.0,
                build_keys=None, nbmin=1e5, nbmax=1e7, gamma=2.0, seed=1, lat_cap=1 << 22):
        n = len(handles)
        H = (ctypes.c_void_p * n)(*[h.handle for h in handles])
        K = (ctypes.c_void_p * n)(*[k.data_ptr() for k in keys_list])
        C = (ctypes.c_uint64 * n)(*[k.numel() for k in keys_list])
        lat = np.empty(int(lat_cap), dtype=np.float64)
        nl, nk, nb, el = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_double()
        self.latency_parts()  # start the record afresh
        rc = lib().mphf_server_loadgen(
            self._p, H, K, C, n, float(rate_hz), float(duration_s), float(bmin), float(bmax),
            out.data_ptr(), out.numel(), float(build_frac),
            build_keys.data_ptr() if build_keys is not None else None,
            build_keys.numel() if build_keys is not None else 0, float(nbmin), float(nbmax),
            float(gamma), int(seed), lat.ctypes.data, lat.size, ctypes.byref(nl), ctypes.byref(nk),
            ctypes.byref(nb), ctypes.byref(el))
        _check(rc, "mphf_server_loadgen")
        m = int(min(nl.value, lat.size))
        return {"latencies": lat[:m].copy(), "lookups": nl.value, "keys": nk.value,
                "builds": nb.value, "elapsed": el.value, "parts": self.latency_parts()}

    def latency_parts(self) -> dict:
        """p50 / p99 seconds of the queue wait, the batch GPU time and the rest
        for the lookups completed since the last call (mphf_server_latency_parts)."""
        p50 = (ctypes.c_double * 3)()
        p99 = (ctypes.c_double * 3)()
        _check(lib().mphf_server_latency_parts(self._p, p50, p99), "mphf_server_latency_parts")
        names = ("queue", "gpu", "rest")
        return {n: {"p50": p50[i], "p99": p99[i]} for i, n in enumerate(names)}


def ceiling(kind: str, buf, n_ops: int, seed: int = 1, width: int = 32, stream=None) -> tuple:
    """One ceiling-measurement launch over the device tensor `buf`:
    kind 'loads' (width 8 or 32 bytes), 'atomics' (result unused) or
    'atomics_ret' (result used).  Returns (accesses performed, ms) from events
    around the launch on the stream."""
    import torch
    st = torch.cuda.current_stream() if stream is None else stream
    sink = torch.zeros(1024, dtype=torch.int64, device=buf.device)
    done = ctypes.c_uint64()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    if kind == "loads":
        rc = lib().mphf_ceiling_random_loads(buf.data_ptr(), buf.numel() * buf.element_size(),
                                             int(width), int(n_ops), int(seed), sink.data_ptr(),
                                             ctypes.byref(done), _stream_ptr(st))
    else:
        rc = lib().mphf_ceiling_random_atomics(buf.data_ptr(), buf.numel(),
                                               1 if kind == "atomics_ret" else 0, int(n_ops),
                                               int(seed), sink.data_ptr(), ctypes.byref(done),
                                               _stream_ptr(st))
    e1.record(st)
    _check(rc, "mphf_ceiling_" + kind)
    e1.synchronize()
    return done.value, e0.elapsed_time(e1)


# ------------------------------------------------- partitioned functions
def route(keys, K: int, part_seed: int, with_src: bool = True, stream=None):
    """Keys grouped by part (mphf_route): (routed, src or None, offsets (K + 1,
    host uint64))."""
    import torch
    keys = _dev_keys(keys)
    n = keys.numel()
    routed = torch.empty(n, dtype=torch.int64, device=keys.device)
    src = torch.empty(n, dtype=torch.int64, device=keys.device) if with_src else None
    off = np.zeros(int(K) + 1, dtype=np.uint64)
    rc = lib().mphf_route(keys.data_ptr() if n else None, n, int(K), int(part_seed) & NOT_FOUND,
                          routed.data_ptr() if n else None,
                          src.data_ptr() if (src is not None and n) else None, off.ctypes.data,
                          _stream_ptr(stream))
    _check(rc, "mphf_route")
    return routed, src, off


def unroute(vals, src, out=None, stream=None):
    """out[src[i]] = vals[i] (mphf_unroute)."""
    import torch
    if out is None:
        out = torch.empty_like(vals)
    n = vals.numel()
    rc = lib().mphf_unroute(vals.data_ptr() if n else None, src.data_ptr() if n else None, n,
                            out.data_ptr() if n else None, _stream_ptr(stream))
    _check(rc, "mphf_unroute")
    return out


def add_offset(vals, offset: int, stream=None):
    """vals += offset where vals is not NOT_FOUND (mphf_add_offset), in place."""
    n = vals.numel()
    rc = lib().mphf_add_offset(vals.data_ptr() if n else None, n, int(offset) & NOT_FOUND,
                               _stream_ptr(stream))
    _check(rc, "mphf_add_offset")
    return vals


class PartitionedMPHF:
    """K independent functions over a hash split of the keys; global index =
    keys in the parts before + index within the part (mphf_build_partitioned)."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle
        K = ctypes.c_uint32()
        _check(lib().mphf_part_info(self._h, ctypes.byref(K), None), "mphf_part_info")
        self.K = K.value
        self.offsets = np.zeros(self.K + 1, dtype=np.uint64)
        _check(lib().mphf_part_info(self._h, ctypes.byref(K), self.offsets.ctypes.data),
               "mphf_part_info")
        self.N = int(self.offsets[-1])

    @classmethod
    def build(cls, keys, K: int, part_seed: int, gamma: float = 2.0, levels: int = 25,
              seed: int = 0, stream=None) -> "PartitionedMPHF":
        keys = _dev_keys(keys)
        h = ctypes.c_void_p()
        rc = lib().mphf_build_partitioned(keys.data_ptr() if keys.numel() else None, keys.numel(),
                                          int(K), int(part_seed) & NOT_FOUND, float(gamma),
                                          int(levels), int(seed) & NOT_FOUND, _stream_ptr(stream),
                                          ctypes.byref(h))
        _check(rc, "mphf_build_partitioned")
        return cls(h)

    def function(self, k: int) -> MPHF:
        p = lib().mphf_part_function(self._h, int(k))
        if not p:
            raise IndexError(k)
        return MPHF(ctypes.c_void_p(p), owner=self)

    def lookup(self, keys, out=None, stream=None):
        import torch
        keys = _dev_keys(keys)
        if out is None:
            out = torch.empty(keys.numel(), dtype=torch.int64, device=keys.device)
        rc = lib().mphf_part_lookup(self._h, keys.data_ptr() if keys.numel() else None,
                                    keys.numel(), out.data_ptr() if keys.numel() else None,
                                    _stream_ptr(stream))
        _check(rc, "mphf_part_lookup")
        return out

    def free(self):
        if self._h is not None and self._h.value:
            lib().mphf_part_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:  # pragma: no cover - interpreter shutdown
            pass


def pool_trim() -> None:
    """Return the library's unused cached device memory to the driver."""
    _check(lib().mphf_pool_trim(), "mphf_pool_trim")


def ceiling_copy(src, dst, stream=None) -> float:
    """One streaming-copy launch src -> dst (device tensors of equal bytes);
    returns its event-timed milliseconds."""
    import torch
    st = torch.cuda.current_stream() if stream is None else stream
    nb = src.numel() * src.element_size()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    rc = lib().mphf_ceiling_copy(src.data_ptr(), dst.data_ptr(), nb, _stream_ptr(st))
    e1.record(st)
    _check(rc, "mphf_ceiling_copy")
    e1.synchronize()
    return e0.elapsed_time(e1)


def launch_count() -> int:
    return lib().mphf_launch_count()


def profile_enable(on: bool = True):
    lib().mphf_profile_enable(1 if on else 0)


def profile_report() -> dict:
    """{kernel name: (launches, total_ms)} of the launches recorded since the last report."""
    buf = ctypes.create_string_buffer(1 << 16)
    _check(lib().mphf_profile_report(buf, len(buf)), "mphf_profile_report")
    out = {}
    for line in buf.value.decode().splitlines():
        name, cnt, ms = line.split()
        out[name] = (int(cnt), float(ms))
    return out


def to_u64(t) -> np.ndarray:
    """A torch int64 tensor (any device) as a numpy uint64 array."""
    return t.detach().cpu().numpy().view(np.uint64)
