"""Partitioned functions (one independent function per part of a hash split
of the keys, Sec. 4.3) on the GPU against the oracle's partitioned mode.

The routing must place every key in its oracle part (offsets equal, each
part's keys equal as a set, the source positions a bijection), scatter back
must invert it, and mphf_build_partitioned + mphf_part_lookup must give the
oracle's global index for every member and non-member, each part's function
being the oracle's function of that part.  DistributedMPHF runs once on a
real NCCL group of one rank.
"""
import ctypes
import os
import socket

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


@pytest.mark.parametrize("n,K", [(0, 3), (1, 1), (5000, 1), (100003, 2), (100003, 7),
                                 (300007, 64), (50000, 1024)])
def test_route_places_every_key_in_its_part(M, n, K):
    keys = inputs.splitmix64_keys(n, 170 + K)
    routed, src, off = M.route(dev(keys), K, 33)
    p = oracle.parts(keys, K, 33)
    want = np.zeros(K + 1, dtype=np.uint64)
    np.cumsum(np.bincount(p.astype(np.int64), minlength=K).astype(np.uint64), out=want[1:])
    assert np.array_equal(off, want)
    r = M.to_u64(routed)
    s = src.cpu().numpy()
    assert np.array_equal(np.sort(s), np.arange(n))
    assert np.array_equal(r, keys[s])
    for k in range(K):
        seg = r[int(off[k]):int(off[k + 1])]
        assert np.array_equal(np.sort(seg), np.sort(keys[p == k]))
    assert np.array_equal(M.to_u64(M.unroute(routed, src)), keys)


def test_add_offset_skips_misses(M):
    v = np.array([0, 5, (1 << 64) - 1, 17, (1 << 64) - 1], dtype=np.uint64)
    t = dev(v)
    M.add_offset(t, 1000)
    assert M.to_u64(t).tolist() == [1000, 1005, (1 << 64) - 1, 1017, (1 << 64) - 1]


@pytest.mark.parametrize("n,K,gamma,levels", [(200003, 1, 2.0, 25), (200003, 2, 2.0, 25),
                                              (300007, 3, 1.0, 25), (300007, 8, 2.0, 3),
                                              (500009, 64, 5.0, 25), (100000, 1024, 2.0, 25),
                                              (35_000_000, 2, 2.0, 25)])
def test_partitioned_function_equals_oracle(M, n, K, gamma, levels):
    # the last case has parts above 2^24 keys: built one by one by mphf_build
    keys = inputs.splitmix64_keys(n, 180 + K)
    P = oracle.PartitionedOracle(keys, K, 44, gamma=gamma, levels=levels, seed=6)
    g = M.PartitionedMPHF.build(dev(keys), K, 44, gamma=gamma, levels=levels, seed=6)
    assert g.K == K and np.array_equal(g.offsets, P.offsets)
    for k in sorted({0, K // 2, K - 1}):
        f, o = g.function(k), P.functions[k]
        assert f.levels() == o.levels()
        assert np.array_equal(f.bits(), o.bits())
        assert np.array_equal(f.fallback(), o.fallback())
    q = np.concatenate([inputs.shuffled(keys, 7), inputs.splitmix64_keys(20000, 181)])
    if n > 10**7:
        q = np.concatenate([keys[inputs.sample_indices(n, 10**6, 8)],
                            inputs.splitmix64_keys(20000, 181)])
    got = M.to_u64(g.lookup(dev(q)))
    assert np.array_equal(got, P.lookup(q))
    if n <= 10**7:
        assert np.array_equal(np.sort(got[:n]), np.arange(n, dtype=np.uint64))
    else:
        out = g.lookup(dev(keys))
        hits = torch.zeros(n, dtype=torch.int32, device="cuda")
        hits.index_add_(0, out, torch.ones_like(out, dtype=torch.int32))
        assert bool((hits == 1).all())


def test_partitioned_rejects_bad_arguments(M):
    L = M.lib()
    h = ctypes.c_void_p()
    k = dev(inputs.splitmix64_keys(100, 190))
    for K in (0, 1025):
        assert L.mphf_build_partitioned(k.data_ptr(), 100, K, 1, 2.0, 25, 0, None,
                                        ctypes.byref(h)) == M.EINVAL
    assert L.mphf_build_partitioned(k.data_ptr(), 100, 4, 1, 0.5, 25, 0, None,
                                    ctypes.byref(h)) == M.EINVAL
    off = np.zeros(3, dtype=np.uint64)
    assert L.mphf_route(k.data_ptr(), 100, 0, 1, k.data_ptr(), None, off.ctypes.data,
                        None) == M.EINVAL
    assert L.mphf_part_lookup(None, k.data_ptr(), 100, k.data_ptr(), None) == M.EINVAL


def test_distributed_one_rank_nccl(M):
    # the multi-GPU wrapper on a real NCCL group of one rank: the one part is
    # the whole key set, so indices equal the plain partitioned function's
    import torch.distributed as dist
    from paper_1702_03154_gb300.distributed import DistributedMPHF
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("nccl", rank=0, world_size=1)
    try:
        keys = inputs.splitmix64_keys(123457, 191)
        d = DistributedMPHF(dev(keys), part_seed=5, gamma=2.0, levels=25, seed=2)
        P = oracle.PartitionedOracle(keys, 1, 5, gamma=2.0, levels=25, seed=2)
        q = np.concatenate([inputs.shuffled(keys, 3), inputs.splitmix64_keys(999, 192)])
        assert np.array_equal(M.to_u64(d.lookup(dev(q))), P.lookup(q))
        assert d.N == keys.size
    finally:
        dist.destroy_process_group()
