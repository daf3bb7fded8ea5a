"""Serving: multi-function lookups and the continuous-batching server.

Every request's result must equal the oracle's (Algorithm 3, the minimal
index of Sec. 2.2.3, on the oracle's own function over the same keys), and be
the same alone (mphf_lookup on its own) and in the mix (coalesced with other
requests, while builds run), exactly.  The multi-function kernel the server
runs (32-bit probe arithmetic) is checked against the oracle in all three
storage layouts, members and non-members.
"""
import threading

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


RESIDENT_SIZES = [1, 37, 4096, 20000, 150001, 600000]


def resident_args(i):
    """gamma, L, seed of resident function i (L = 2 leaves a large fallback)."""
    return (2.0 if i % 2 else 1.0), (25 if i != 3 else 2), i


@pytest.fixture(scope="module")
def resident(M):
    hs, ks = [], []
    for i, n in enumerate(RESIDENT_SIZES):
        k = dev(inputs.splitmix64_keys(n, 300 + i))
        g, L, seed = resident_args(i)
        hs.append(M.MPHF.build(k, gamma=g, levels=L, seed=seed))
        ks.append(k)
    return hs, ks


@pytest.fixture(scope="module")
def oracles():
    os_ = []
    for i, n in enumerate(RESIDENT_SIZES):
        g, L, seed = resident_args(i)
        os_.append(oracle.build(inputs.splitmix64_keys(n, 300 + i), gamma=g, levels=L, seed=seed))
    return os_


def test_lookup_multi_equals_alone(M, resident, oracles):
    hs, ks = resident
    rng = np.random.default_rng(1)
    reqs = []
    for t in range(40):
        i = int(rng.integers(len(hs)))
        n = ks[i].numel()
        b = int(rng.integers(0, min(n, 5000) + 1))
        o = int(rng.integers(0, n - b + 1))
        reqs.append((i, ks[i][o:o + b]))
    # non-member keys too
    reqs.append((4, dev(inputs.splitmix64_keys(1000, 999))))
    outs = M.lookup_multi([hs[i] for i, _ in reqs], [k for _, k in reqs])
    for (i, k), o in zip(reqs, outs):
        alone = hs[i].lookup(k) if k.numel() else torch.empty(0, dtype=torch.int64, device="cuda")
        assert torch.equal(o, alone)
        assert np.array_equal(M.to_u64(o), oracles[i].lookup(M.to_u64(k)))


def test_server_results_same_alone_and_in_mix(M, resident, oracles):
    hs, ks = resident
    hk = [M.to_u64(k) for k in ks]
    srv = M.Server(max_batch_keys=1 << 18, max_batch_reqs=256, max_inflight=3, build_workers=2,
                   mem_reserve=1 << 30)
    rng = np.random.default_rng(5)
    plan = []
    for t in range(300):
        i = int(rng.integers(len(hs)))
        n = ks[i].numel()
        b = int(np.exp(rng.uniform(0, np.log(min(n, 100000)))))
        b = max(1, min(b, n))
        o = int(rng.integers(0, n - b + 1))
        plan.append((i, o, b))
    build_keys = [dev(inputs.splitmix64_keys(n, 700 + j)) for j, n in enumerate((1000, 120000))]
    outs = [torch.full((b,), -7, dtype=torch.int64, device="cuda") for (_, _, b) in plan]
    torch.cuda.synchronize()
    rids = [None] * len(plan)
    bids = []

    def submit(lo, hi):
        for t in range(lo, hi):
            i, o, b = plan[t]
            rids[t] = srv.submit_lookup(hs[i], ks[i][o:o + b], outs[t])

    th = [threading.Thread(target=submit, args=(a, a + 100)) for a in (0, 100, 200)]
    for t in th:
        t.start()
    for bk in build_keys:
        bids.append(srv.submit_build(bk, gamma=2.0, levels=25, seed=3))
    for t in th:
        t.join()
    for t, rid in enumerate(rids):
        st, lat, _ = srv.wait(rid)
        assert st == M.OK and lat >= 0
    built = []
    for rid in bids:
        st, lat, h = srv.wait(rid)
        assert st == M.OK and h is not None
        built.append(h)
    stats = srv.stats()
    assert stats["requests"] == len(plan)
    assert stats["batches"] < len(plan)        # requests were coalesced
    srv.close()
    for t, (i, o, b) in enumerate(plan):
        assert torch.equal(outs[t], hs[i].lookup(ks[i][o:o + b])), t
        assert np.array_equal(M.to_u64(outs[t]), oracles[i].lookup(hk[i][o:o + b])), t
    for j, (n, h) in enumerate(zip((1000, 120000), built)):
        kh = inputs.splitmix64_keys(n, 700 + j)
        ref = oracle.build(kh, gamma=2.0, levels=25, seed=3)
        assert np.array_equal(h.bits(), ref.bits())
        assert np.array_equal(h.rank(), ref.rank())
        assert np.array_equal(M.to_u64(h.lookup(dev(kh))), ref.lookup(kh))


def test_server_build_waits_for_memory(M):
    # a reserve larger than the device keeps every build waiting
    srv = M.Server(build_workers=1, mem_reserve=1 << 50)
    k = dev(inputs.splitmix64_keys(10000, 5))
    rid = srv.submit_build(k)
    with pytest.raises(M.MPHFError) as e:
        srv.wait(rid, timeout=0.5)
    assert e.value.code == M.ETIMEOUT
    srv.close()


def test_server_loadgen_reports_latencies(M, resident):
    hs, ks = resident
    srv = M.Server(max_batch_keys=1 << 20, max_batch_reqs=1024, max_inflight=3, build_workers=1)
    out = torch.empty(1 << 20, dtype=torch.int64, device="cuda")
    bk = dev(inputs.splitmix64_keys(200000, 11))
    r = srv.loadgen(hs[2:], ks[2:], rate_hz=2000.0, duration_s=0.5, bmin=1, bmax=20000, out=out,
                    build_frac=0.01, build_keys=bk, nbmin=1e4, nbmax=2e5)
    srv.close()
    assert r["lookups"] > 500
    assert r["latencies"].size == r["lookups"]
    assert np.all(r["latencies"] > 0)


@pytest.mark.parametrize("layouts", [(32, 32, 32, 32), (64, 64, 64, 64), (8, 8, 8, 8),
                                     (32, 64, 8, 64)])
def test_multi_function_kernel_equals_oracle_every_layout(M, layouts):
    # The server's kernel: one launch over requests to several functions,
    # 32-bit probe arithmetic (every function here is far below 2^36 bits),
    # grouped by storage layout.  Requests are members (shuffled), members
    # answered by the fallback (L = 2), non-members, empty and tiny batches,
    # and batches large enough to be cut into warp chunks.
    specs = [(300000, 2.0, 25), (70001, 1.0, 2), (5000, 5.0, 25), (1_000_003, 2.0, 25)]
    hs, qs, want = [], [], []
    for i, ((n, g, L), lay) in enumerate(zip(specs, layouts)):
        kh = inputs.splitmix64_keys(n, 400 + i)
        o = oracle.build(kh, gamma=g, levels=L, seed=20 + i)
        h = M.MPHF.build(dev(kh), gamma=g, levels=L, seed=20 + i)
        h.set_layout(lay)
        q = np.concatenate([inputs.shuffled(kh, 30 + i), inputs.splitmix64_keys(3001, 500 + i)])
        hs.append(h)
        qs.append(q)
        want.append(o.lookup(q))
    assert hs[1].num_fallback > 0
    # many requests per function, of mixed sizes (0, 1, 17, ..., whole)
    rng = np.random.default_rng(sum(layouts))
    rh, rk, rw = [], [], []
    for t in range(60):
        i = int(rng.integers(len(hs)))
        b = min(int(rng.choice([0, 1, 17, 2048, 40000, qs[i].size])), qs[i].size)
        o = int(rng.integers(0, qs[i].size - b + 1))
        rh.append(hs[i])
        rk.append(dev(qs[i][o:o + b]))
        rw.append(want[i][o:o + b])
    outs = M.lookup_multi(rh, rk)
    for o, w in zip(outs, rw):
        assert np.array_equal(M.to_u64(o), w)
