"""Batched construction vs per-set plain builds vs the CPU oracle.

mphf_build_batched must give every set exactly the function mphf_build (and
the oracle) gives it: same level sizes, A bits, rank checkpoints, fallback and
indices.
"""
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


def same(g, o):
    assert g.N == o.N
    assert g.levels() == o.levels()
    assert g.num_fallback == o.num_fallback
    assert np.array_equal(g.bits(), o.bits())
    assert np.array_equal(g.rank(), o.rank())
    assert np.array_equal(g.fallback(), o.fallback())


def make_sets(S, lo, hi, seed, extra_sizes=()):
    sizes = list(inputs.log_uniform_sizes(S, lo, hi, seed)) + list(extra_sizes)
    off = inputs.set_offsets(np.array(sizes, dtype=np.int64))
    keys = np.concatenate([inputs.splitmix64_keys(int(n), 7, start=int(off[i]))
                           for i, n in enumerate(sizes)]) if sizes else np.zeros(0, np.uint64)
    return keys, off


@pytest.mark.parametrize("gamma,levels", [(2.0, 25), (1.0, 25), (5.0, 25), (1.0, 3)])
def test_batched_matches_oracle_per_set(M, gamma, levels):
    keys, off = make_sets(48, 1, 80000, 7 + int(gamma), extra_sizes=(0, 1, 2, 16384, 16385, 70001))
    hs = M.build_batched(dev(keys), off, gamma=gamma, levels=levels, seed=4)
    assert len(hs) == off.size - 1
    for s, g in enumerate(hs):
        k = keys[off[s]:off[s + 1]]
        o = oracle.build(k, gamma=gamma, levels=levels, seed=4)
        same(g, o)
        if k.size:
            assert np.array_equal(M.to_u64(g.lookup(dev(k))), o.lookup(k))
            assert g.build_path in (1, 2, 3)


def test_device_offsets_through_the_c_abi(M):
    # mphf_build_batched takes the S + 1 offsets in device memory; the
    # functions equal the host-offset call's and the oracle's.
    import ctypes
    keys, off = make_sets(20, 1, 50000, 13, extra_sizes=(0, 16385))
    kd = dev(keys)
    od = torch.from_numpy(off.view(np.int64)).cuda()
    L = M.lib()
    S = off.size - 1
    arr = (ctypes.c_void_p * S)()
    rc = L.mphf_build_batched(kd.data_ptr(), od.data_ptr(), S, 2.0, 25, 5,
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), arr)
    assert rc == M.OK
    hs = [M.MPHF(ctypes.c_void_p(arr[i])) for i in range(S)]
    hh = M.build_batched(kd, off, gamma=2.0, levels=25, seed=5)
    hd = M.build_batched(kd, od, gamma=2.0, levels=25, seed=5)
    for s in range(S):
        k = keys[off[s]:off[s + 1]]
        o = oracle.build(k, gamma=2.0, levels=25, seed=5)
        for g in (hs[s], hh[s], hd[s]):
            same(g, o)
    # decreasing offsets are refused, and no handle comes back
    bad = off.copy()
    bad[3], bad[4] = bad[4], bad[3]
    arr2 = (ctypes.c_void_p * S)()
    rc = L.mphf_build_batched(kd.data_ptr(), torch.from_numpy(bad.view(np.int64)).cuda().data_ptr(),
                              S, 2.0, 25, 5, None, arr2)
    assert rc == M.EINVAL and all(arr2[i] is None for i in range(S))


def test_batched_equals_plain_builds(M):
    keys, off = make_sets(32, 1000, 300000, 11)
    kd = dev(keys)
    hs = M.build_batched(kd, off, gamma=2.0, levels=25, seed=9)
    for s, g in enumerate(hs):
        p = M.MPHF.build(kd[int(off[s]):int(off[s + 1])], gamma=2.0, levels=25, seed=9)
        assert g.levels() == p.levels()
        assert np.array_equal(g.bits(), p.bits())
        assert np.array_equal(g.rank(), p.rank())
        assert g.bits_per_key() == p.bits_per_key()


def test_batched_overflow_rebuilds_sets(M):
    keys, off = make_sets(16, 20000, 200000, 13)
    try:
        M.batched_debug_config(0.4)
        hs = M.build_batched(dev(keys), off, gamma=2.0, levels=25, seed=1)
    finally:
        M.batched_debug_config(1.0)
    assert any(g.build_path != 3 for g in hs)
    for s, g in enumerate(hs):
        k = keys[off[s]:off[s + 1]]
        o = oracle.build(k, gamma=2.0, levels=25, seed=1)
        same(g, o)


def test_batched_reports_duplicates(M):
    keys, off = make_sets(8, 1000, 50000, 17)
    keys[int(off[3]) + 5] = keys[int(off[3]) + 9]
    with pytest.raises(M.MPHFError) as e:
        M.build_batched(dev(keys), off, gamma=2.0, levels=25, seed=0)
    assert e.value.code == M.EDUPLICATE


def test_batched_repeated_calls_replay_identically(M):
    keys, off = make_sets(40, 1000, 200000, 19)
    kd = dev(keys)
    a = M.build_batched(kd, off, gamma=2.0, levels=25, seed=3)
    b = M.build_batched(kd, off, gamma=2.0, levels=25, seed=3)   # replays the recorded graph
    for x, y in zip(a, b):
        assert np.array_equal(x.bits(), y.bits())
        assert np.array_equal(x.rank(), y.rank())


def test_autotune_does_not_change_results(M):
    keys, off = make_sets(24, 1000, 150000, 23)
    kd = dev(keys)
    before = M.build_batched(kd, off, gamma=2.0, levels=25, seed=5)
    ms = M.autotune_batched(kd, off, gamma=2.0, levels=25, seed=5)
    assert ms > 0
    after = M.build_batched(kd, off, gamma=2.0, levels=25, seed=5)
    for x, y in zip(before, after):
        assert np.array_equal(x.bits(), y.bits())
        assert np.array_equal(x.rank(), y.rank())


def test_batched_config4_full_size_sampled(M):
    # 4096 sets, sizes log-uniform in [1e3, 1e6] (seed 7), gamma = 2, L = 25, as
    # the benchmark times it: every set's lookups are a bijection (checked on the
    # GPU), and 12 sampled sets match the oracle exactly.
    sizes = inputs.log_uniform_sizes(4096, 1e3, 1e6, 7)
    off = inputs.set_offsets(sizes)
    from paper_1702_03154_gb300 import mphf
    keys_d = mphf.keygen(int(off[-1]), 7)
    hs = M.build_batched(keys_d, off, gamma=2.0, levels=25, seed=0)
    out = torch.empty_like(keys_d)
    for s, g in enumerate(hs):
        a, b = int(off[s]), int(off[s + 1])
        g.lookup(keys_d[a:b], out=out[a:b])
    # bijection per set: out[a:b] is a permutation of 0..n-1
    seg = torch.repeat_interleave(torch.arange(4096, device="cuda"),
                                  torch.from_numpy(sizes).cuda())
    base = torch.from_numpy(off[:-1].astype(np.int64)).cuda()
    glob = out + base[seg]
    assert int(out.min()) >= 0
    hit = torch.zeros(int(off[-1]), dtype=torch.int32, device="cuda")
    hit.index_add_(0, glob, torch.ones_like(glob, dtype=torch.int32))
    assert bool((hit == 1).all())
    rng = np.random.default_rng(3)
    keys_h = None
    for s in sorted(rng.choice(4096, 12, replace=False).tolist()):
        a, b = int(off[s]), int(off[s + 1])
        k = M.to_u64(keys_d[a:b])
        o = oracle.build(k, gamma=2.0, levels=25, seed=0)
        same(hs[s], o)


@pytest.mark.parametrize("pmax,bset,tail", [(4096, 1, 4096), (32768, 16, 4096), (262144, 2048, 8192),
                                            (65536, 64, 8192)])
def test_every_tuning_gives_the_oracle_result(M, pmax, bset, tail):
    # the tuning moves bucket widths, buckets per set and the tail block shape;
    # the function stays the paper's (narrow choices overflow and re-build)
    keys, off = make_sets(30, 2000, 120000, 29)
    S, total = len(off) - 1, int(off[-1])
    M.batched_set_tuning(S, total, pmax, bset, tail)
    assert M.batched_tuning(S, total) == {"bucket_width_max": pmax, "buckets_per_set_max": bset,
                                          "tail_keys": tail}
    hs = M.build_batched(dev(keys), off, gamma=2.0, levels=25, seed=8)
    for s in (0, 7, 18, 29):
        k = keys[int(off[s]):int(off[s + 1])]
        o = oracle.build(k, gamma=2.0, levels=25, seed=8)
        assert np.array_equal(hs[s].bits(), o.bits())
        assert np.array_equal(hs[s].fallback(), o.fallback())
        assert np.array_equal(M.to_u64(hs[s].lookup(dev(k))), o.lookup(k))
    M.batched_set_tuning(S, total, 131072, 64, 8192)


def test_autotune_choice_is_reported(M):
    keys, off = make_sets(16, 1000, 90000, 31)
    S, total = len(off) - 1, int(off[-1])
    M.autotune_batched(dev(keys), off, gamma=2.0, levels=25, seed=1)
    t = M.batched_tuning(S, total)
    assert t["bucket_width_max"] in (32768, 65536, 131072, 262144)
    assert t["buckets_per_set_max"] in (16, 64) and t["tail_keys"] in (4096, 8192)


def test_bad_tuning_is_refused(M):
    for args in ((4095, 64, 8192), (3 * 4096, 64, 8192), (524288, 64, 8192), (65536, 0, 8192),
                 (65536, 4096, 8192), (65536, 64, 2048)):
        with pytest.raises(M.MPHFError) as e:
            M.batched_set_tuning(10, 10**6, *args)
        assert e.value.code == M.EINVAL
