"""Serving: multi-function lookups and the continuous-batching server.

Every request's result must be the same alone (mphf_lookup on its own) and
in the mix (coalesced with other requests, while builds run), exactly.
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


@pytest.fixture(scope="module")
def resident(M):
    sizes = [1, 37, 4096, 20000, 150001, 600000]
    hs, ks = [], []
    for i, n in enumerate(sizes):
        k = dev(inputs.splitmix64_keys(n, 300 + i))
        hs.append(M.MPHF.build(k, gamma=2.0 if i % 2 else 1.0, levels=25 if i != 3 else 2, seed=i))
        ks.append(k)
    return hs, ks


def test_lookup_multi_equals_alone(M, resident):
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


def test_server_results_same_alone_and_in_mix(M, resident):
    hs, ks = resident
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
    for bk, h in zip(build_keys, built):
        ref = oracle.build(M.to_u64(bk), gamma=2.0, levels=25, seed=3)
        assert np.array_equal(h.bits(), ref.bits())
        assert np.array_equal(h.rank(), ref.rank())


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
