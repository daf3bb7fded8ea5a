"""The 1e10-key configuration: properties that hold at any size.

N = 1e10 keys generated on the device by the SplitMix64 stream of seed 4
(80 GB), gamma = 2, L = 25.  The CPU oracle cannot build a function this
large in test time, so the checks are: every key's index, in chunks, lands on
a distinct value of [0, N) (a counter per index on the device); each level
places (1 - 1/m_d)^(n_d - 1) of its keys within 6 sigma; the total bits and
bits/key match gamma e^{1/gamma} N and 1.125 gamma e^{1/gamma} (Sec. 2.3,
Sec. 3.1) within 0.5%; placed keys plus fallback add up to N.
"""
import math

import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N = 10**10


def test_config3_1e10_properties():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, total = torch.cuda.mem_get_info()
    if free < 240 * 2**30:
        pytest.skip(f"needs ~240 GB of free device memory, {free / 2**30:.0f} GB free")
    from paper_1702_03154_gb300 import mphf
    keys = mphf.keygen(N, 4)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    h = mphf.MPHF.build(keys, gamma=2.0, levels=25, seed=0)
    e1.record()
    torch.cuda.synchronize()
    print(f"build of 1e10 keys: {e0.elapsed_time(e1) / 1e3:.3f} s "
          f"({N / (e0.elapsed_time(e1) / 1e3) / 1e9:.2f} Gkeys/s), {h.bits_per_key():.4f} bits/key")
    lv = h.levels()
    sizes = h.level_sizes()
    assert sizes[0] == N
    # per-level placed fraction
    for d, (n_d, m_d, off_d, _) in enumerate(lv[:6]):
        p = (1.0 - 1.0 / m_d) ** (n_d - 1)
        placed = sizes[d] - sizes[d + 1]
        assert abs(placed - n_d * p) < 6 * math.sqrt(n_d * p * (1 - p)) + 1, d
    g = 2.0
    assert abs(h.total_bits / N - g * math.exp(1 / g)) / (g * math.exp(1 / g)) < 0.005
    assert abs(h.bits_per_key() - 1.125 * g * math.exp(1 / g)) < 0.02
    # every index distinct, in [0, N)
    hits = torch.zeros(N, dtype=torch.int32, device="cuda")
    one = None
    chunk = 500_000_000
    for a in range(0, N, chunk):
        idx = h.lookup(keys[a:a + chunk])
        assert int(idx.min()) >= 0 and int(idx.max()) < N
        if one is None or one.numel() != idx.numel():
            one = torch.ones(idx.numel(), dtype=torch.int32, device="cuda")
        hits.index_add_(0, idx, one)
        del idx
    assert bool((hits == 1).all())
    del hits
    # 1e9 member lookups at random positions (the configuration's query set)
    sel = torch.randint(0, N, (10**9,), device="cuda", generator=torch.Generator(device="cuda").manual_seed(5))
    q = keys[sel]
    del sel
    out = torch.empty_like(q)
    h.lookup(q, out=out)  # warm
    e0.record()
    h.lookup(q, out=out)
    e1.record()
    torch.cuda.synchronize()
    print(f"1e9 random member lookups: {e0.elapsed_time(e1):.1f} ms "
          f"({1e9 / (e0.elapsed_time(e1) / 1e3) / 1e9:.2f} Gkeys/s)")
    assert int(out.min()) >= 0 and int(out.max()) < N
    del q, out
    total_placed = N - h.num_fallback
    assert total_placed + h.num_fallback == N
    # The same function built without storing any key (Sec. 3.4, second
    # strategy; Sec. 4.4 streams generated keys the same way): equal, bit for bit.
    import time
    import numpy as np
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g2 = mphf.MPHF.build_generated(N, 4, 0, gamma=2.0, levels=25, seed=0)
    t1 = time.perf_counter()
    print(f"generated-key build of 1e10 keys: {t1 - t0:.2f} s")
    assert g2.levels() == lv and g2.total_bits == h.total_bits
    assert g2.num_fallback == h.num_fallback
    assert np.array_equal(g2.rank(), h.rank())
    q = keys[::997]
    assert torch.equal(g2.lookup(q), h.lookup(q))
