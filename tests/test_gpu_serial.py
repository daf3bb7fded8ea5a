"""Serialized images: a loaded function is the built one, bit for bit.

A function saved with mphf_serialize and loaded with mphf_deserialize must
answer every query exactly as before (and as the oracle), and must expose the
same A, checkpoints and fallback.  Damaged images are rejected with
MPHF_EINVAL: a flipped payload byte (checksum), a truncated buffer, a wrong
magic, and a header whose checksum is valid but whose level table breaks the
sizing rule m_d = max(64, ceil64(gamma n_d)) of Sec. 2.2.4.
"""
import struct

import numpy as np
import pytest

import oracle
from paper_1702_03154_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MASK = (1 << 64) - 1


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_03154_gb300 import mphf
    mphf.lib()
    return mphf


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def same(g, o):
    assert g.N == o.N and g.levels() == o.levels() and g.total_bits == o.total_bits
    assert g.num_fallback == o.num_fallback
    assert np.array_equal(g.bits(), o.bits())
    assert np.array_equal(g.rank(), o.rank())
    assert np.array_equal(g.fallback(), o.fallback())


@pytest.mark.parametrize("n,gamma,levels", [(100003, 2.0, 25), (50000, 1.0, 2), (1, 5.0, 25),
                                            (2 * 10**6, 2.0, 25)])
def test_round_trip(M, n, gamma, levels):
    keys = inputs.splitmix64_keys(n, 71)
    o = oracle.build(keys, gamma=gamma, levels=levels, seed=12)
    g = M.MPHF.build(dev(keys), gamma=gamma, levels=levels, seed=12)
    img = g.to_bytes()
    h = M.MPHF.from_bytes(img)
    assert h.build_path == 4
    same(h, o)
    q = np.concatenate([keys, inputs.splitmix64_keys(5000, 72)])
    want = o.lookup(q)
    assert np.array_equal(M.to_u64(h.lookup(dev(q))), want)
    assert np.array_equal(M.to_u64(g.lookup(dev(q))), want)
    assert h.to_bytes() == img  # the image of a loaded function is the same image


def test_empty_function(M):
    g = M.MPHF.build(torch.empty(0, dtype=torch.int64, device="cuda"), 2.0, 25, 0)
    h = M.MPHF.from_bytes(g.to_bytes())
    assert h.N == 0 and h.num_levels == 0
    assert M.to_u64(h.lookup(dev(np.array([5, 6], dtype=np.uint64)))).tolist() == [MASK, MASK]


def test_batched_handle_and_file(M, tmp_path):
    sizes = np.array([1000, 20000, 3333], dtype=np.uint64)
    keys = inputs.splitmix64_keys(int(sizes.sum()), 73)
    offs = inputs.set_offsets(sizes)
    hs = M.build_batched(dev(keys), offs, gamma=2.0, levels=25, seed=2)
    for i, hb in enumerate(hs):
        k = keys[int(offs[i]):int(offs[i + 1])]
        path = tmp_path / f"f{i}.bbh"
        hb.save(str(path))
        h = M.MPHF.load(str(path))
        same(h, oracle.build(k, gamma=2.0, levels=25, seed=2))
        assert np.array_equal(M.to_u64(h.lookup(dev(k))), M.to_u64(hb.lookup(dev(k))))


def _checksum(payload: bytes) -> int:
    # SplitMix64-finalizer chain over the payload's 8-byte words, then the count
    def mix(z):
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        return z ^ (z >> 31)
    h = 0x6a09e667f3bcc908
    words = np.frombuffer(payload, dtype=np.uint64)
    for w in words.tolist():
        h = mix((h + w) & MASK)
    return mix(h ^ len(words))


def test_damaged_images_are_rejected(M):
    keys = inputs.splitmix64_keys(30000, 74)
    g = M.MPHF.build(dev(keys), gamma=2.0, levels=25, seed=3)
    img = bytearray(g.to_bytes())
    # the checksum covers the payload: recomputing it must give the stored one
    assert struct.unpack_from("<Q", img, 88)[0] == _checksum(bytes(img[128:]))

    def rejected(b):
        with pytest.raises(M.MPHFError) as e:
            M.MPHF.from_bytes(bytes(b))
        assert e.value.code == M.EINVAL

    flipped = bytearray(img)
    flipped[len(img) // 2] ^= 0x10
    rejected(flipped)
    rejected(img[:-8])
    rejected(img[:100])
    bad_magic = bytearray(img)
    bad_magic[0:8] = b"NOTBBHGB"
    rejected(bad_magic)
    # level 0's m_d off by 64 bits with a recomputed (valid) checksum
    bad_m = bytearray(img)
    m0 = struct.unpack_from("<Q", bad_m, 128 + 8)[0]
    struct.pack_into("<Q", bad_m, 128 + 8, m0 + 64)
    struct.pack_into("<Q", bad_m, 88, _checksum(bytes(bad_m[128:])))
    rejected(bad_m)
    # and the untouched image still loads
    h = M.MPHF.from_bytes(bytes(img))
    assert np.array_equal(M.to_u64(h.lookup(dev(keys))), M.to_u64(g.lookup(dev(keys))))
