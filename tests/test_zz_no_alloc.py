"""The allocation-free rank-table entry point agrees with the library's own.

mphf_rank_table_noalloc exists for callers that may not allocate device
memory (code being recorded into a CUDA graph, serving loops on a fixed
memory budget, hosts whose allocator owns the device memory).  Called through
the C ABI on the A bits of a function built by mphf_build, its checkpoints
must equal those mphf_build produced (mphf_copy_rank) and the oracle's rank
table for the same keys, exactly, on two calls in a row (the second reuses
the library's fixed scratch array).  A second case fills the scratch to its
last entry: random words just under the 2^27-word limit (65536 blocks of
partial sums), against a host prefix sum of popcounts.  This file is
collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1702_03154_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_rank_table_matches_build():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_03154_gb300 import mphf
    L = mphf.lib()
    keys = inputs.splitmix64_keys(3_000_000, 83)
    kd = torch.from_numpy(keys.view(np.int64)).cuda()
    h = mphf.MPHF.build(kd, gamma=2.0, levels=25, seed=1)
    words = h.bits()
    want = h.rank()
    o = oracle.build(keys, gamma=2.0, levels=25, seed=1)
    assert np.array_equal(o.rank(), want)
    assert np.array_equal(o.bits(), words)
    nrank = want.size
    assert nrank == (words.size + 7) // 8
    wd = torch.from_numpy(words.view(np.int64)).cuda()
    stream = torch.cuda.current_stream()
    for call in range(2):
        out = torch.full((2 * nrank,), -1, dtype=torch.int64, device="cuda")
        total = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        rc = L.mphf_rank_table_noalloc(wd.data_ptr(), words.size, out.data_ptr(),
                                       total.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
        assert rc == mphf.OK, L.mphf_strerror(rc)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint64)
        assert np.array_equal(got[0::2], want), f"call {call}: checkpoints differ"
        # in-block prefix counts: ones of words 0..k-1 of each 512-bit block
        pc = np.unpackbits(words.view(np.uint8)).reshape(-1, 64).sum(axis=1)
        pc = np.concatenate([pc, np.zeros(8 * nrank - pc.size, dtype=pc.dtype)]).reshape(nrank, 8)
        pre = np.cumsum(pc, axis=1)[:, :7].astype(np.uint64)
        rel = np.zeros(nrank, dtype=np.uint64)
        for k in range(1, 8):
            rel |= pre[:, k - 1] << np.uint64(9 * (k - 1))
        assert np.array_equal(got[1::2], rel), f"call {call}: in-block counts differ"
        assert int(total.item()) == keys.size - o.num_fallback


def _popcount64(w):
    if hasattr(np, "bitwise_count"):
        return np.bitwise_count(w)
    lut = np.array([bin(i).count("1") for i in range(256)], dtype=np.uint8)
    return lut[w.view(np.uint8)].reshape(-1, 8).sum(axis=1, dtype=np.uint8)


def test_noalloc_rank_table_at_its_limit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_03154_gb300 import mphf
    L = mphf.lib()
    nwords = (1 << 27) - 5          # 2^24 blocks, the last one ragged: 65536 CTAs
    rng = np.random.Generator(np.random.PCG64(84))
    words = rng.integers(0, 2**63, size=nwords, dtype=np.int64).view(np.uint64)
    words[::3] &= np.uint64(0x00FF00FF00FF00FF)  # uneven densities
    nrank = (nwords + 7) // 8
    pc = np.zeros(8 * nrank, dtype=np.uint64)
    pc[:nwords] = _popcount64(words)
    blk = pc.reshape(nrank, 8).sum(axis=1)
    want = np.zeros(nrank, dtype=np.uint64)
    np.cumsum(blk[:-1], out=want[1:])
    wd = torch.from_numpy(words.view(np.int64)).cuda()
    out = torch.empty(2 * nrank, dtype=torch.int64, device="cuda")
    total = torch.empty(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    for call in range(2):
        out.fill_(-1)
        total.fill_(-1)
        rc = L.mphf_rank_table_noalloc(wd.data_ptr(), nwords, out.data_ptr(), total.data_ptr(),
                                       ctypes.c_void_p(stream.cuda_stream))
        assert rc == mphf.OK, L.mphf_strerror(rc)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint64)
        assert np.array_equal(got[0::2], want), f"call {call}"
        assert int(total.item()) == int(pc.sum())


def test_noalloc_rejects_oversize_input():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_03154_gb300 import mphf
    L = mphf.lib()
    buf = torch.zeros(16, dtype=torch.int64, device="cuda")
    rc = L.mphf_rank_table_noalloc(buf.data_ptr(), (1 << 27) + 8, buf.data_ptr(), None, None)
    assert rc == mphf.EINVAL
