"""CUDA path vs the CPU oracle, bit for bit.

The GPU build must give the oracle's level sizes and seeds, the same A bits,
rank checkpoints and fallback keys, and the same index for every key (members
and non-members).  All comparisons are exact: the method is integer-only and
its result does not depend on the order in which keys are processed.
"""
import numpy as np
import pytest

import oracle
from paper_1702_03154_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U64 = (1 << 64) - 1


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_03154_gb300 import mphf
    mphf.lib()
    return mphf


def dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def assert_same_structure(g, o):
    assert g.N == o.N
    assert g.num_levels == o.num_levels
    assert g.levels() == o.levels()
    assert g.total_bits == o.total_bits
    assert g.num_fallback == o.num_fallback
    assert np.array_equal(g.bits(), o.bits())
    assert np.array_equal(g.rank(), o.rank())
    assert np.array_equal(g.fallback(), o.fallback())
    assert g.bits_per_key() == pytest.approx(o.bits_per_key(), abs=0, rel=0)


def check(M, keys, gamma, levels, seed, queries=None):
    o = oracle.build(keys, gamma=gamma, levels=levels, seed=seed)
    g = M.MPHF.build(dev(keys), gamma=gamma, levels=levels, seed=seed)
    assert_same_structure(g, o)
    q = keys if queries is None else queries
    out = M.to_u64(g.lookup(dev(q)))
    assert np.array_equal(out, o.lookup(q))
    return g, o


def test_config1_full_parity(M):
    # N = 1e6 keys = SplitMix64 outputs 0..N-1 of seed 1, gamma = 2, L = 25.
    keys = inputs.splitmix64_keys(10**6, 1)
    g, o = check(M, keys, 2.0, 25, 0)
    out = M.to_u64(g.lookup(dev(keys)))
    assert np.array_equal(np.sort(out), np.arange(keys.size, dtype=np.uint64))
    others = inputs.splitmix64_keys(200000, 101)
    assert np.array_equal(M.to_u64(g.lookup(dev(others))), o.lookup(others))


@pytest.mark.parametrize("n", [1, 2, 3, 63, 64, 65, 127, 4095, 4096, 4097, 8191, 12345, 100003])
@pytest.mark.parametrize("gamma", [1.0, 1.5, 2.0, 5.0])
def test_ragged_sizes(M, n, gamma):
    keys = inputs.splitmix64_keys(n, 7 + n)
    check(M, keys, gamma, 25, n)


@pytest.mark.parametrize("levels", [1, 2, 3, 5])
def test_small_level_budgets_exercise_fallback(M, levels):
    keys = inputs.splitmix64_keys(50000, 17)
    g, o = check(M, keys, 1.0, levels, 3)
    assert g.num_fallback > 0


def test_large_fallback_uses_global_sort(M):
    # L = 1 at gamma = 1 leaves ~63% of the keys in the fallback (> 4096).
    keys = inputs.splitmix64_keys(100000, 23)
    g, o = check(M, keys, 1.0, 1, 9)
    assert g.num_fallback > 4096


def test_misaligned_key_pointers(M):
    keys = inputs.splitmix64_keys(100001, 29)
    o = oracle.build(keys[1:], gamma=2.0, levels=25, seed=4)
    buf = dev(keys)
    g = M.MPHF.build(buf[1:], gamma=2.0, levels=25, seed=4)   # 8-byte aligned only
    assert_same_structure(g, o)
    out = torch.empty(keys.size, dtype=torch.int64, device="cuda")
    g.lookup(buf[1:], out=out[1:])
    assert np.array_equal(M.to_u64(out[1:]), o.lookup(keys[1:]))


def test_order_independence(M):
    keys = inputs.splitmix64_keys(300000, 31)
    a = M.MPHF.build(dev(keys), gamma=1.0, levels=25, seed=5)
    b = M.MPHF.build(dev(inputs.shuffled(keys, 9)), gamma=1.0, levels=25, seed=5)
    assert a.levels() == b.levels()
    assert np.array_equal(a.bits(), b.bits())
    assert np.array_equal(a.rank(), b.rank())
    assert np.array_equal(a.fallback(), b.fallback())


def test_repeated_builds_are_identical(M):
    keys = inputs.splitmix64_keys(500000, 37)
    a = M.MPHF.build(dev(keys), gamma=2.0, levels=25, seed=1)
    for _ in range(3):
        b = M.MPHF.build(dev(keys), gamma=2.0, levels=25, seed=1)
        assert np.array_equal(a.bits(), b.bits())
        assert np.array_equal(a.rank(), b.rank())


def test_empty_and_single(M):
    g = M.MPHF.build(torch.empty(0, dtype=torch.int64, device="cuda"), 2.0, 25, 0)
    assert g.num_levels == 0 and g.total_bits == 0 and g.num_fallback == 0
    assert g.bits_per_key() == 0.0
    q = dev(np.array([1, 2, 3], dtype=np.uint64))
    assert M.to_u64(g.lookup(q)).tolist() == [U64] * 3
    g1 = M.MPHF.build(dev(np.array([12345], dtype=np.uint64)), 2.0, 25, 0)
    assert M.to_u64(g1.lookup(dev(np.array([12345], dtype=np.uint64)))).tolist() == [0]


@pytest.mark.parametrize("n,levels", [(1000, 25), (100000, 1)])
def test_duplicates_are_reported(M, n, levels):
    keys = inputs.splitmix64_keys(n, 41)
    keys[n // 2] = keys[3]
    with pytest.raises(M.MPHFError) as e:
        M.MPHF.build(dev(keys), gamma=1.0, levels=levels, seed=0)
    assert e.value.code == M.EDUPLICATE
    # the library is still usable afterwards
    check(M, inputs.splitmix64_keys(1000, 43), 2.0, 25, 0)


def test_invalid_arguments(M):
    k = dev(inputs.splitmix64_keys(10, 1))
    for gamma, levels in ((0.9, 25), (float("nan"), 25), (2.0, 0), (2.0, 65)):
        with pytest.raises(M.MPHFError) as e:
            M.MPHF.build(k, gamma=gamma, levels=levels)
        assert e.value.code == M.EINVAL


def test_host_buffer_entry_points(M):
    keys = inputs.splitmix64_keys(200001, 47)
    o = oracle.build(keys, gamma=2.0, levels=25, seed=6)
    g = M.MPHF.build_host(keys, gamma=2.0, levels=25, seed=6)
    assert_same_structure(g, o)
    pinned = torch.from_numpy(keys.view(np.int64)).pin_memory()
    out = g.lookup_host(pinned)
    assert np.array_equal(out, o.lookup(keys))


@pytest.mark.parametrize("pinned", [True, False])
def test_host_entry_points_chunked(M, pinned):
    # Past 4 Mi keys the host entry points stream the batch in chunks (copy of
    # chunk c+1 beside the work on chunk c); n leaves a ragged last chunk.
    n = (1 << 22) + 12345
    keys = inputs.splitmix64_keys(n, 48)
    q = np.concatenate([inputs.shuffled(keys, 5)[: n - 1000],
                        inputs.splitmix64_keys(1000, 49)])
    o = oracle.build(keys, gamma=2.0, levels=25, seed=8)
    src = torch.from_numpy(keys.view(np.int64)).pin_memory() if pinned else keys
    g = M.MPHF.build_host(src, gamma=2.0, levels=25, seed=8)
    assert g.build_path == 1
    assert_same_structure(g, o)
    qs = torch.from_numpy(q.view(np.int64)).pin_memory() if pinned else q
    out = np.empty(n, dtype=np.uint64)
    if pinned:
        ot = torch.empty(n, dtype=torch.int64).pin_memory()
        g.lookup_host(qs, out=ot.numpy().view(np.uint64))
        out = ot.numpy().view(np.uint64).copy()
    else:
        g.lookup_host(qs, out=out)
    assert np.array_equal(out, o.lookup(q))


@pytest.mark.parametrize("path,cap_scale", [(1, 1.0), (0, 0.5)])
def test_host_build_chunked_unbucketed_path(M, path, cap_scale):
    # The unbucketed construction reads every key at once: the streamed copy
    # must be complete before it starts, whether it was chosen up front
    # (path 1) or after the bucketed partition overflowed (cap_scale 0.5).
    n = (1 << 22) + 777
    keys = inputs.splitmix64_keys(n, 50)
    o = oracle.build(keys, gamma=1.0, levels=25, seed=9)
    M.debug_config(path, cap_scale)
    try:
        g = M.MPHF.build_host(keys, gamma=1.0, levels=25, seed=9)
    finally:
        M.debug_config(0, 1.0)
    assert g.build_path == 2
    assert_same_structure(g, o)


@pytest.mark.parametrize("cap_scale", [1.0, 0.3])
def test_host_build_grouped_level0(M, cap_scale):
    # Keys streamed from host memory into a build whose level 0 is grouped by
    # slab (with the slab capacities scaled down the ranges overflow and level
    # 0 is grouped again with exact counts): the function and the indices of
    # the oracle.
    n = (1 << 22) + 777
    keys = inputs.splitmix64_keys(n, 63)
    q = np.concatenate([inputs.shuffled(keys, 9), inputs.splitmix64_keys(5000, 64)])
    o = oracle.build(keys, gamma=2.0, levels=25, seed=16)
    M.debug_config(1, cap_scale)
    M.debug_slabs(16, 0)
    try:
        g, out = M.MPHF.build_lookup_host(keys, q, gamma=2.0, levels=25, seed=16)
    finally:
        M.debug_slabs()
        M.debug_config(0, 1.0)
    assert g.build_path == 2
    assert_same_structure(g, o)
    assert np.array_equal(out, o.lookup(q))


def test_host_lookup_chunked_empty_function(M):
    g = M.MPHF.build_host(np.empty(0, dtype=np.uint64))
    q = inputs.splitmix64_keys((1 << 22) + 5, 51)
    out = g.lookup_host(q)
    assert np.all(out == np.uint64(U64))


def test_device_keygen_matches_generator(M):
    for n, seed, start in ((1, 0, 0), (1000, 1, 0), (100003, 4, 12345)):
        got = M.to_u64(M.keygen(n, seed, start))
        assert np.array_equal(got, inputs.splitmix64_keys(n, seed, start=start))


@pytest.mark.parametrize("gamma", [1.0, 2.0, 5.0])
def test_config2_shape_parity_1e7(M, gamma):
    # The N = 1e8 workload's shape at 1e7 keys: full structure + every lookup.
    keys = inputs.splitmix64_keys(10**7, 2)
    q = inputs.shuffled(keys, 3)
    check(M, keys, gamma, 25, 0, queries=q)


@pytest.mark.parametrize("gamma", [2.0, 1.0, 5.0])
def test_config2_full_size(M, gamma):
    # N = 1e8, L = 25, as the benchmark times it (gamma = 2; 1 and 5 as its
    # sweep does; at gamma = 1 about 1e3 keys reach the fallback): the full
    # structure (levels, A, rank, fallback) and every one of the 1e8 indices,
    # queried in shuffled order, against the oracle; 1e6 non-members too.
    N = 10**8
    keys = inputs.splitmix64_keys(N, 2)
    o = oracle.build(keys, gamma=gamma, levels=25, seed=0)
    kd = dev(keys)
    g = M.MPHF.build(kd, gamma=gamma, levels=25, seed=0)
    if gamma == 1.0:
        assert g.num_fallback > 0
    assert_same_structure(g, o)
    del kd
    q = inputs.shuffled(keys, 3)
    del keys
    out = M.to_u64(g.lookup(dev(q)))
    assert np.array_equal(out, o.lookup(q))
    assert np.array_equal(np.sort(out), np.arange(N, dtype=np.uint64))
    del out, q
    others = inputs.splitmix64_keys(10**6, 103)
    assert np.array_equal(M.to_u64(g.lookup(dev(others))), o.lookup(others))


@pytest.mark.parametrize("n,gamma,levels", [(10**6, 2.0, 25), (300001, 1.0, 25), (300001, 5.0, 25),
                                            (200000, 1.0, 3), (20000, 2.0, 25)])
def test_unbucketed_path_matches(M, n, gamma, levels):
    keys = inputs.splitmix64_keys(n, 53)
    o = oracle.build(keys, gamma=gamma, levels=levels, seed=2)
    try:
        M.debug_config(path=1)
        g = M.MPHF.build(dev(keys), gamma=gamma, levels=levels, seed=2)
    finally:
        M.debug_config(path=0)
    assert g.build_path == 2
    assert_same_structure(g, o)
    assert np.array_equal(M.to_u64(g.lookup(dev(keys))), o.lookup(keys))


def test_default_path_is_bucketed(M):
    keys = inputs.splitmix64_keys(10**6, 59)
    g = M.MPHF.build(dev(keys), gamma=2.0, levels=25, seed=0)
    assert g.build_path == 1


@pytest.mark.parametrize("n", [10**6, 100000])
def test_bucket_overflow_falls_back_with_identical_results(M, n):
    keys = inputs.splitmix64_keys(n, 61)
    o = oracle.build(keys, gamma=2.0, levels=25, seed=3)
    try:
        M.debug_config(path=0, cap_scale=0.5)
        g = M.MPHF.build(dev(keys), gamma=2.0, levels=25, seed=3)
    finally:
        M.debug_config(path=0, cap_scale=1.0)
    assert g.build_path == 2
    assert_same_structure(g, o)
    assert np.array_equal(M.to_u64(g.lookup(dev(keys))), o.lookup(keys))


def test_many_duplicates_are_reported(M):
    # 5000 copies of one key overflow a bucket: the unbucketed path reports them.
    keys = inputs.splitmix64_keys(200000, 67)
    keys[:5000] = keys[5000]
    with pytest.raises(M.MPHFError) as e:
        M.MPHF.build(dev(keys), gamma=2.0, levels=25, seed=0)
    assert e.value.code == M.EDUPLICATE


@pytest.mark.parametrize("kind", ["sequential", "stride_2_40", "high_bit", "extremes"])
def test_structured_keys(M, kind):
    # the method hashes every key, so structured (non-random) keys must give
    # exactly the oracle's function too
    n = 200003
    j = np.arange(n, dtype=np.uint64)
    if kind == "sequential":
        keys = j
    elif kind == "stride_2_40":
        keys = j << np.uint64(40)
    elif kind == "high_bit":
        keys = j | np.uint64(1 << 63)
    else:
        keys = np.concatenate([np.array([0, (1 << 64) - 1, 1 << 63, (1 << 63) - 1], dtype=np.uint64),
                               inputs.splitmix64_keys(n - 4, 120)])
    check(M, keys, 2.0, 25, 11)


@pytest.mark.parametrize("gamma", [1.0, 7.5, 100.0])
def test_extreme_gamma(M, gamma):
    keys = inputs.splitmix64_keys(50021, 121)
    g, o = check(M, keys, gamma, 25, 12)
    # at large gamma almost every key is placed at level 0
    if gamma == 100.0:
        assert g.level_sizes()[1] < keys.size * 0.02


def test_large_fallback_at_scale(M):
    # L = 1 at gamma = 1: ~63% of 2e6 keys go to the sorted fallback
    keys = inputs.splitmix64_keys(2 * 10**6, 122)
    g, o = check(M, keys, 1.0, 1, 13)
    assert g.num_fallback > 10**6


@pytest.mark.parametrize("n,nq,pinned", [((1 << 22) + 12345, (1 << 22) + 999, True),
                                         ((1 << 22) + 3, 5000, False),
                                         (200001, (1 << 22) + 77, True),
                                         (777, 1000, False)])
def test_build_lookup_host_is_build_then_lookup(M, n, nq, pinned):
    # The pipelined call (queries copied behind the keys while the levels are
    # built, lookups chunk by chunk) gives the function and the indices of the
    # two separate calls, chunked or not on either side.
    keys = inputs.splitmix64_keys(n, 52)
    extra = inputs.splitmix64_keys(nq, 53)
    q = np.concatenate([inputs.shuffled(keys, 6)[: nq // 2], extra[: nq - min(nq // 2, n)]])
    q = q[:nq]
    o = oracle.build(keys, gamma=2.0, levels=25, seed=10)
    ks = torch.from_numpy(keys.view(np.int64)).pin_memory() if pinned else keys
    qs = torch.from_numpy(q.view(np.int64)).pin_memory() if pinned else q
    if pinned:
        ot = torch.empty(q.size, dtype=torch.int64).pin_memory()
        g, _ = M.MPHF.build_lookup_host(ks, qs, out=ot.numpy().view(np.uint64), gamma=2.0,
                                        levels=25, seed=10)
        out = ot.numpy().view(np.uint64).copy()
    else:
        g, out = M.MPHF.build_lookup_host(ks, qs, gamma=2.0, levels=25, seed=10)
    assert_same_structure(g, o)
    assert np.array_equal(out, o.lookup(q))


def test_build_lookup_host_edges(M):
    # no keys: every query misses; no queries: just the function
    g, out = M.MPHF.build_lookup_host(np.empty(0, dtype=np.uint64),
                                      inputs.splitmix64_keys(1000, 54))
    assert g.N == 0 and np.all(out == np.uint64(U64))
    keys = inputs.splitmix64_keys(5000, 55)
    g, out = M.MPHF.build_lookup_host(keys, np.empty(0, dtype=np.uint64), seed=3)
    assert out.size == 0
    assert_same_structure(g, oracle.build(keys, gamma=2.0, levels=25, seed=3))
    # duplicates: reported, no function returned
    dup = np.concatenate([keys, keys[:10]])
    with pytest.raises(M.MPHFError) as e:
        M.MPHF.build_lookup_host(dup, keys)
    assert e.value.code == M.EDUPLICATE


@pytest.mark.parametrize("gamma,levels,shift", [(2.0, 25, 12), (1.0, 25, 10), (5.0, 25, 14),
                                                (1.0, 3, 12), (2.0, 25, 8), (2.0, 25, 6)])
def test_unbucketed_slab_grouping(M, gamma, levels, shift):
    # The unbucketed path groups a level's keys by slabs of 2^shift positions
    # before filling it (all levels here: threshold 0).  Shift 8 gives levels
    # 0 and 1 more slabs than threads (the multisplit whose threads own
    # several slabs) and the later levels fewer (one slab per thread); shift 6
    # gives more slabs than a multisplit takes, so level 0 is left ungrouped.
    keys = inputs.splitmix64_keys(200001, 56)
    q = np.concatenate([inputs.shuffled(keys, 7), inputs.splitmix64_keys(5000, 57)])
    o = oracle.build(keys, gamma=gamma, levels=levels, seed=11)
    M.debug_config(1, 1.0)
    M.debug_slabs(shift, 0)
    try:
        g = M.MPHF.build(dev(keys), gamma=gamma, levels=levels, seed=11)
        dup = np.concatenate([keys, keys[:7]])
        with pytest.raises(M.MPHFError) as e:
            M.MPHF.build(dev(dup), gamma=gamma, levels=levels, seed=11)
        assert e.value.code == M.EDUPLICATE
    finally:
        M.debug_slabs()
        M.debug_config(0, 1.0)
    assert g.build_path == 2
    assert_same_structure(g, o)
    assert np.array_equal(M.to_u64(g.lookup(dev(q))), o.lookup(q))


def test_grouped_level0_many_equal_keys(M):
    # 40000 copies of one key push |F_1| past the bound that the grouped
    # level 0 sizes F_1 by: the compaction of level 0 runs again into an
    # exactly sized buffer, and the duplicates are reported; the same keys
    # without the copies give the oracle's function.
    keys = inputs.splitmix64_keys(300007, 62)
    o = oracle.build(keys, gamma=2.0, levels=25, seed=15)
    dup = np.concatenate([keys, np.full(40000, keys[11], dtype=np.uint64)])
    M.debug_config(1, 1.0)
    M.debug_slabs(20, 0)
    try:
        with pytest.raises(M.MPHFError) as e:
            M.MPHF.build(dev(dup), gamma=2.0, levels=25, seed=15)
        assert e.value.code == M.EDUPLICATE
        g = M.MPHF.build(dev(keys), gamma=2.0, levels=25, seed=15)
    finally:
        M.debug_slabs()
        M.debug_config(0, 1.0)
    assert g.build_path == 2
    assert_same_structure(g, o)
    assert np.array_equal(M.to_u64(g.lookup(dev(keys))), o.lookup(keys))


@pytest.mark.parametrize("cap_scale", [1.0, 0.3])
def test_unbucketed_grouping_overflow_redo(M, cap_scale):
    # Fine slabs take fixed-capacity ranges; a range that overflows (capacity
    # scaled down here, or thousands of copies of one key) makes the level
    # redo its grouping with exact counts: same function, duplicates reported.
    keys = inputs.splitmix64_keys(300007, 60)
    o = oracle.build(keys, gamma=2.0, levels=25, seed=14)
    M.debug_config(1, cap_scale)
    M.debug_slabs(20, 0)
    try:
        g = M.MPHF.build(dev(keys), gamma=2.0, levels=25, seed=14)
        dup = np.concatenate([keys, np.full(5000, keys[3], dtype=np.uint64)])
        with pytest.raises(M.MPHFError) as e:
            M.MPHF.build(dev(dup), gamma=2.0, levels=25, seed=14)
        assert e.value.code == M.EDUPLICATE
    finally:
        M.debug_slabs()
        M.debug_config(0, 1.0)
    assert g.build_path == 2
    assert_same_structure(g, o)
    assert np.array_equal(M.to_u64(g.lookup(dev(keys))), o.lookup(keys))


def test_unbucketed_slab_grouping_at_scale(M):
    # 1.5e8 keys at gamma 2: level 0's hit/collision array (75 MB) is past the
    # default threshold, so the unbucketed path groups it into 3 slabs and
    # fills each fine slab in shared memory.  Both paths against the oracle:
    # levels, A, rank, fallback; every index a bijection on the GPU, and 2e6
    # sampled members plus non-members against the oracle.
    N = 150_000_000
    keys = inputs.splitmix64_keys(N, 58)
    o = oracle.build(keys, gamma=2.0, levels=25, seed=12)
    kd = dev(keys)
    a = M.MPHF.build(kd, gamma=2.0, levels=25, seed=12)
    M.debug_config(1, 1.0)
    try:
        b = M.MPHF.build(kd, gamma=2.0, levels=25, seed=12)
    finally:
        M.debug_config(0, 1.0)
    assert a.build_path == 1 and b.build_path == 2
    assert_same_structure(b, o)
    assert_same_structure(a, o)
    for g in (a, b):
        out = g.lookup(kd)
        hits = torch.zeros(N, dtype=torch.int32, device="cuda")
        assert int(out.min()) >= 0 and int(out.max()) < N
        hits.index_add_(0, out, torch.ones_like(out, dtype=torch.int32))
        assert bool((hits == 1).all())
        del out, hits
    idx = inputs.sample_indices(N, 2 * 10**6, 6)
    q = np.concatenate([keys[idx], inputs.splitmix64_keys(10**5, 104)])
    want = o.lookup(q)
    assert np.array_equal(M.to_u64(b.lookup(dev(q))), want)
    assert np.array_equal(M.to_u64(a.lookup(dev(q))), want)
