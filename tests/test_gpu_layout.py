"""Rank sampling: 32-byte (default), 64-byte ("minirank") sectors, 8-byte units.

Re-storing a function in the other sector size must leave every index, the
plain A and the paper's checkpoints unchanged; only the size moves, and it
moves the way the paper's two settings do (Sec. 3.1, Sec. 4.3: one counter
per 512 or per 1024 bits; at gamma = 1 the printed sizes are 3.1 and 2.9
bits/key).
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1702_03154_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_03154_gb300 import mphf
    mphf.lib()
    return mphf


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


@pytest.mark.parametrize("gamma,levels", [(1.0, 25), (2.0, 25), (5.0, 25), (1.0, 3)])
@pytest.mark.parametrize("nbytes", [64, 8])
def test_relayout_keeps_every_index(M, gamma, levels, nbytes):
    keys = inputs.splitmix64_keys(400009, 111)
    o = oracle.build(keys, gamma=gamma, levels=levels, seed=7)
    g = M.MPHF.build(dev(keys), gamma=gamma, levels=levels, seed=7)
    assert g.sector_bytes == 32
    q = np.concatenate([keys, inputs.splitmix64_keys(20000, 112)])
    want = o.lookup(q)
    small_before = g.device_bytes()
    g.set_layout(nbytes)
    assert g.sector_bytes == nbytes
    assert np.array_equal(g.bits(), o.bits())
    assert np.array_equal(g.rank(), o.rank())
    assert np.array_equal(g.fallback(), o.fallback())
    assert np.array_equal(M.to_u64(g.lookup(dev(q))), want)
    M_bits = o.total_bits
    if nbytes == 64:
        # minirank: the paper's accounting with 1024-bit counters; one 32-bit
        # count per 15 A words, one 64-bit count per 2^24 sectors
        assert g.bits_per_key() == pytest.approx(o.bits_per_key_sampled(1024), rel=1e-12)
        assert g.device_bytes() < small_before
        nsect = -(-(M_bits // 32) // 15)
        want_bytes = 64 * nsect + 8 * -(-nsect // 2**24)
    else:
        # 8-byte units of 48 bits of A; one 64-bit count per 1024 units; the
        # paper's default accounting
        assert g.bits_per_key() == pytest.approx(o.bits_per_key(), rel=1e-12)
        assert g.device_bytes() > small_before
        nunits = -(-M_bits // 48)
        want_bytes = 8 * nunits + 8 * -(-nunits // 1024)
    assert g.device_bytes() == want_bytes + 8 * g.num_fallback
    g.set_layout(32)
    assert g.sector_bytes == 32 and g.device_bytes() == small_before
    assert np.array_equal(M.to_u64(g.lookup(dev(q))), want)
    assert g.bits_per_key() == pytest.approx(o.bits_per_key(), rel=1e-12)


def test_minirank_sizes_match_the_paper(M, golden_dir):
    t = json.load(open(os.path.join(golden_dir, "table1_bits_per_key.json")))
    keys = inputs.splitmix64_keys(10**6, 113)
    g = M.MPHF.build(dev(keys), gamma=1.0, levels=25, seed=0)
    rows = {(r["gamma"], r["rank_block"]): r["bits_per_key"] for r in t["rows"]}
    tol = t["printed_precision"] + 0.01
    assert abs(g.bits_per_key() - rows[(1.0, 512)]) <= tol
    g.set_layout(64)
    assert abs(g.bits_per_key() - rows[(1.0, 1024)]) <= tol


@pytest.mark.parametrize("nbytes", [64, 8])
def test_relayout_image_round_trip(M, nbytes):
    keys = inputs.splitmix64_keys(123457, 114)
    g = M.MPHF.build(dev(keys), gamma=2.0, levels=25, seed=1)
    g.set_layout(nbytes)
    h = M.MPHF.from_bytes(g.to_bytes())
    assert h.sector_bytes == nbytes
    assert np.array_equal(h.bits(), g.bits()) and np.array_equal(h.rank(), g.rank())
    assert torch.equal(h.lookup(dev(keys)), g.lookup(dev(keys)))


def test_multi_lookup_mixes_layouts(M):
    sets = [inputs.splitmix64_keys(n, 115 + i) for i, n in enumerate((5000, 70000, 300, 123456))]
    hs = [M.MPHF.build(dev(k), gamma=2.0, levels=25, seed=3) for k in sets]
    hs[1].set_layout(64)
    hs[2].set_layout(8)
    hs[3].set_layout(64)
    qs = [dev(np.concatenate([k, inputs.splitmix64_keys(777, 130 + i)])) for i, k in enumerate(sets)]
    outs = M.lookup_multi(hs, qs)
    for h, q, o in zip(hs, qs, outs):
        assert torch.equal(o, h.lookup(q))


def test_batched_handle_takes_its_own_arrays(M):
    sizes = np.array([3000, 40000, 1234], dtype=np.uint64)
    keys = inputs.splitmix64_keys(int(sizes.sum()), 116)
    offs = inputs.set_offsets(sizes)
    hs = M.build_batched(dev(keys), offs, gamma=2.0, levels=25, seed=4)
    before = [M.to_u64(h.lookup(dev(keys[int(offs[i]):int(offs[i + 1])]))) for i, h in enumerate(hs)]
    hs[1].set_layout(64)
    hs[0].free()  # the shared arena must outlive its other users
    for i in (1, 2):
        k = keys[int(offs[i]):int(offs[i + 1])]
        assert np.array_equal(M.to_u64(hs[i].lookup(dev(k))), before[i])
        o = oracle.build(k, gamma=2.0, levels=25, seed=4)
        assert np.array_equal(hs[i].bits(), o.bits())


def test_bad_sector_size_is_refused(M):
    g = M.MPHF.build(dev(inputs.splitmix64_keys(100, 117)))
    for b in (0, 16, 48, 128, 4):
        with pytest.raises(M.MPHFError) as e:
            g.set_layout(b)
        assert e.value.code == M.EINVAL


def test_wide_position_kernels_every_layout(M):
    # The kernels with 64-bit position arithmetic (taken on their own only by
    # functions past 2^32-bit levels or 2^36 bits of A) give the same indices
    # in every layout, single- and multi-function.
    keys = inputs.splitmix64_keys(300007, 118)
    q = np.concatenate([inputs.shuffled(keys, 9), inputs.splitmix64_keys(9999, 119)])
    o = oracle.build(keys, gamma=2.0, levels=25, seed=13)
    want = o.lookup(q)
    hs = [M.MPHF.build(dev(keys), gamma=2.0, levels=25, seed=13) for _ in range(3)]
    hs[1].set_layout(64)
    hs[2].set_layout(8)
    M.debug_lookup_wide(True)
    try:
        for h in hs:
            assert np.array_equal(M.to_u64(h.lookup(dev(q))), want)
        outs = M.lookup_multi(hs, [dev(q)] * 3)
    finally:
        M.debug_lookup_wide(False)
    for out in outs:
        assert np.array_equal(M.to_u64(out), want)
