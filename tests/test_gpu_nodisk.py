"""Construction without stored key sets (Sec. 3.4 second strategy, Sec. 4.5).

Re-reading every key at each level and asking the levels already built
whether it was placed there yields exactly F_d, so the function must be the
oracle's (and the default build's) bit for bit, whatever keep_fraction says
about when F_d is finally stored.  The generated variant streams the keys of
mphf_keygen and must equal a build over those keys.
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
    assert g.N == o.N and g.levels() == o.levels() and g.total_bits == o.total_bits
    assert g.num_fallback == o.num_fallback
    assert np.array_equal(g.bits(), o.bits())
    assert np.array_equal(g.rank(), o.rank())
    assert np.array_equal(g.fallback(), o.fallback())


@pytest.mark.parametrize("gamma", [1.0, 2.0, 5.0])
@pytest.mark.parametrize("keep", [0.0, 0.02, 1.0])
def test_nodisk_matches_oracle(M, gamma, keep):
    keys = inputs.splitmix64_keys(300007, 101)
    o = oracle.build(keys, gamma=gamma, levels=25, seed=4)
    g = M.MPHF.build_nodisk(dev(keys), gamma=gamma, levels=25, seed=4, keep_fraction=keep)
    assert g.build_path == 5
    same(g, o)
    q = np.concatenate([keys[::3], inputs.splitmix64_keys(3000, 102)])
    assert np.array_equal(M.to_u64(g.lookup(dev(q))), o.lookup(q))


@pytest.mark.parametrize("levels,keep", [(1, 0.0), (3, 0.0), (3, 0.5), (5, 1.0)])
def test_nodisk_fallback_paths(M, levels, keep):
    # few levels at gamma = 1 leave many keys for the sorted fallback
    keys = inputs.splitmix64_keys(60000, 103)
    o = oracle.build(keys, gamma=1.0, levels=levels, seed=5)
    g = M.MPHF.build_nodisk(dev(keys), gamma=1.0, levels=levels, seed=5, keep_fraction=keep)
    assert g.num_fallback > 0
    same(g, o)
    assert np.array_equal(M.to_u64(g.lookup(dev(keys))), o.lookup(keys))


@pytest.mark.parametrize("n,key_seed,key_start", [(1, 9, 0), (4097, 9, 123), (10**6, 4, 5 * 10**6)])
def test_generated_matches_oracle(M, n, key_seed, key_start):
    keys = inputs.splitmix64_keys(n, key_seed, start=key_start)
    o = oracle.build(keys, gamma=2.0, levels=25, seed=6)
    g = M.MPHF.build_generated(n, key_seed, key_start, gamma=2.0, levels=25, seed=6)
    same(g, o)
    assert np.array_equal(M.to_u64(g.lookup(dev(keys))), o.lookup(keys))


def test_generated_equals_default_build_at_1e8(M):
    n = 10**8
    keys = M.keygen(n, 2)
    a = M.MPHF.build(keys, gamma=2.0, levels=25, seed=0)
    b = M.MPHF.build_generated(n, 2, 0, gamma=2.0, levels=25, seed=0)
    assert a.levels() == b.levels() and a.total_bits == b.total_bits
    assert np.array_equal(a.bits(), b.bits())
    assert np.array_equal(a.rank(), b.rank())
    q = keys[::97]
    assert torch.equal(a.lookup(q), b.lookup(q))


def test_nodisk_empty_duplicates_and_arguments(M):
    g = M.MPHF.build_nodisk(torch.empty(0, dtype=torch.int64, device="cuda"))
    assert g.N == 0 and g.num_levels == 0
    keys = inputs.splitmix64_keys(20000, 104)
    keys[777] = keys[5]
    with pytest.raises(M.MPHFError) as e:
        M.MPHF.build_nodisk(dev(keys), gamma=2.0, levels=25, keep_fraction=0.0)
    assert e.value.code == M.EDUPLICATE
    for keep in (-0.1, 1.5, float("nan")):
        with pytest.raises(M.MPHFError) as e:
            M.MPHF.build_nodisk(dev(keys[:10]), keep_fraction=keep)
        assert e.value.code == M.EINVAL
