"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that ``include/*.h`` declares (no compute calls here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(mphf_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_1702_03154_gb300 import build_ext
    return build_ext.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for core in ("mphf_build", "mphf_lookup", "mphf_bits_per_key", "mphf_free"):
        assert core in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_error_text_without_gpu(libpath):
    from paper_1702_03154_gb300 import mphf
    L = mphf.lib()
    assert L.mphf_strerror(mphf.EDUPLICATE) == b"duplicate keys"
    assert L.mphf_strerror(mphf.EINVAL) == b"invalid argument"
    assert L.mphf_abi_version() == 2


def test_argument_validation_without_gpu(libpath):
    # Rejected before any CUDA call is made.
    from paper_1702_03154_gb300 import mphf
    L = mphf.lib()
    h = ctypes.c_void_p()
    for gamma, levels in ((0.5, 25), (float("nan"), 25), (float("inf"), 25), (2.0, 0), (2.0, 65)):
        assert L.mphf_build(8, 3, gamma, levels, 0, None, ctypes.byref(h)) == mphf.EINVAL
        assert h.value is None
    assert L.mphf_build(None, 3, 2.0, 25, 0, None, ctypes.byref(h)) == mphf.EINVAL
    assert L.mphf_build(8, 3, 2.0, 25, 0, None, None) == mphf.EINVAL
    assert L.mphf_lookup(None, 8, 1, 8, None) == mphf.EINVAL
    assert L.mphf_bits_per_key(None) == 0.0
    L.mphf_free(None)
    lv = ctypes.c_uint32(7)
    assert L.mphf_num_levels(None, ctypes.byref(lv)) == mphf.EINVAL and lv.value == 7
    outs = (ctypes.c_void_p * 2)()
    assert L.mphf_build_batched(8, None, 2, 2.0, 25, 0, None, outs) == mphf.EINVAL
    assert L.mphf_build_batched(8, 12, 2, 2.0, 25, 0, None, outs) == mphf.EINVAL  # misaligned
    assert L.mphf_build_batched(8, 16, 0, 2.0, 25, 0, None, outs) == mphf.EINVAL
    assert L.mphf_build_batched_host_offsets(8, None, 2, 2.0, 25, 0, None, outs) == mphf.EINVAL


def test_oracle_and_cuda_sources_share_nothing():
    # The oracle is plain C with no include of the CUDA sources and vice versa.
    osrc = open(os.path.join(ROOT, "oracle", "mphf_oracle.c")).read()
    assert "#include \"" not in osrc
    for f in glob.glob(os.path.join(ROOT, "paper_1702_03154_gb300", "csrc", "*")):
        assert "oracle" not in open(f).read().lower(), f
    for f in glob.glob(os.path.join(ROOT, "paper_1702_03154_gb300", "*.py")):
        txt = open(f).read()
        assert "import oracle" not in txt and "from oracle" not in txt, f


def test_new_entry_points_validate_without_gpu(libpath):
    # Host-side argument checks of the later entry points (no CUDA call made).
    from paper_1702_03154_gb300 import mphf
    L = mphf.lib()
    h = ctypes.c_void_p()
    # build + lookup from host buffers
    assert L.mphf_build_lookup_host(8, 3, 2.0, 25, 0, 8, 1, 8, None, None) == mphf.EINVAL
    for gamma, levels in ((0.5, 25), (float("nan"), 25), (2.0, 0), (2.0, 65)):
        assert L.mphf_build_lookup_host(8, 3, gamma, levels, 0, 8, 1, 8, None,
                                        ctypes.byref(h)) == mphf.EINVAL
        assert h.value is None
    assert L.mphf_build_lookup_host(None, 3, 2.0, 25, 0, 8, 1, 8, None,
                                    ctypes.byref(h)) == mphf.EINVAL
    assert L.mphf_build_lookup_host(8, 3, 2.0, 25, 0, None, 1, 8, None,
                                    ctypes.byref(h)) == mphf.EINVAL
    assert L.mphf_build_lookup_host(8, 3, 2.0, 25, 0, 8, 1, None, None,
                                    ctypes.byref(h)) == mphf.EINVAL
    # batched tuning: values outside what the kernels take are refused
    for args in ((4095, 64, 8192), (3 * 4096, 64, 8192), (524288, 64, 8192), (65536, 0, 8192),
                 (65536, 4096, 8192), (65536, 64, 1000)):
        assert L.mphf_batched_set_tuning(10, 10**6, *args) == mphf.EINVAL
    v = [ctypes.c_uint64() for _ in range(3)]
    assert L.mphf_batched_tuning(7, 12345, *[ctypes.byref(x) for x in v]) == mphf.EINVAL
    assert (v[0].value, v[1].value, v[2].value) == (131072, 64, 8192)  # the defaults
    assert L.mphf_batched_set_tuning(7, 12345, 65536, 16, 4096) == mphf.OK
    assert L.mphf_batched_tuning(7, 12345, *[ctypes.byref(x) for x in v]) == mphf.OK
    assert (v[0].value, v[1].value, v[2].value) == (65536, 16, 4096)
    assert L.mphf_batched_set_tuning(7, 12345, 131072, 64, 8192) == mphf.OK
    # test hooks
    assert L.mphf_debug_slabs(5, 0) == mphf.EINVAL and L.mphf_debug_slabs(30, 0) == mphf.EINVAL
    assert L.mphf_debug_slabs(27, 64 << 20) == mphf.OK
    assert L.mphf_debug_size_level(1000, 2.0, 0, *[ctypes.byref(x) for x in v]) == mphf.EINVAL
    assert L.mphf_debug_level1_bound(1000, 0.5, 608, *[ctypes.byref(x) for x in v]) == mphf.EINVAL
