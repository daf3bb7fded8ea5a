"""The 1e10-key configuration: the oracle on windows of level 0, and
properties that hold at any size.

N = 1e10 keys generated on the device by the SplitMix64 stream of seed 4
(80 GB), gamma = 2, L = 25.  The CPU oracle cannot build a function this
large in test time (its byte-per-bit arrays alone would take ~110 GB and its
single-threaded build most of an hour), so:

* oracle parity on windows of level 0: the host draws all 1e10 keys with the
  shared generator and keeps those whose level-0 position falls in three
  windows of 2^22 positions (the start, the middle and the end of A_0); the
  oracle's ArrayFill of each window must equal the GPU's A_0 there, word for
  word, and the oracle's rank inside the window must give the GPU's index of
  every key placed there (exactly for the first window, which starts A; up to
  the window's one common offset -- the ones before it -- for the others);
* every key's index, in chunks, lands on a distinct value of [0, N) (a
  counter per index on the device); each level places (1 - 1/m_d)^(n_d - 1)
  of its keys within 6 sigma; the total bits and bits/key match
  gamma e^{1/gamma} N and 1.125 gamma e^{1/gamma} (Sec. 2.3, Sec. 3.1) within
  0.5%; placed keys plus fallback add up to N.
"""
import math
import os
import sys
import time

import numpy as np
import pytest

import oracle

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import oracle_windows  # noqa: E402

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N = 10**10
KEY_SEED = 4
WIN = 1 << 22
U64MAX = np.uint64((1 << 64) - 1)


def windows_of(m0):
    mid = (m0 // 2) // 64 * 64 + 64 * 1001  # not a multiple of 2^22: any word offset
    return [(0, WIN), (mid, WIN), (m0 - WIN, WIN)]


def test_config3_1e10_properties():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, total = torch.cuda.mem_get_info()
    if free < 240 * 2**30:
        pytest.skip(f"needs ~240 GB of free device memory, {free / 2**30:.0f} GB free")
    from paper_1702_03154_gb300 import mphf
    # level 0 as the oracle defines it (Sec. 2.2.4 size, level-seeded hash)
    s0 = oracle.level_seed(0, 0)
    m0 = oracle.level_bits(N, 2.0)
    wins = windows_of(m0)
    t_sel = time.perf_counter()
    sel = oracle_windows.start_selection(N, KEY_SEED, s0, m0, wins)

    keys = mphf.keygen(N, KEY_SEED)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    h = mphf.MPHF.build(keys, gamma=2.0, levels=25, seed=0)
    e1.record()
    torch.cuda.synchronize()
    print(f"build of 1e10 keys: {e0.elapsed_time(e1) / 1e3:.3f} s "
          f"({N / (e0.elapsed_time(e1) / 1e3) / 1e9:.2f} Gkeys/s), {h.bits_per_key():.4f} bits/key")
    mphf.pool_trim()  # the build's cached scratch back to the driver: the checks below need room
    lv = h.levels()
    sizes = h.level_sizes()
    assert sizes[0] == N
    assert lv[0] == (N, m0, 0, s0)
    # per-level placed fraction
    for d, (n_d, m_d, off_d, _) in enumerate(lv[:6]):
        p = (1.0 - 1.0 / m_d) ** (n_d - 1)
        placed = sizes[d] - sizes[d + 1]
        assert abs(placed - n_d * p) < 6 * math.sqrt(n_d * p * (1 - p)) + 1, d
    g = 2.0
    assert abs(h.total_bits / N - g * math.exp(1 / g)) / (g * math.exp(1 / g)) < 0.005
    assert abs(h.bits_per_key() - 1.125 * g * math.exp(1 / g)) < 0.02

    # the oracle on windows of level 0
    words = h.bits()
    selected = oracle_windows.finish_selection(sel)
    print(f"host selection of the window keys over 1e10 keys: {time.perf_counter() - t_sel:.1f} s "
          f"({[s.size for s in selected]} keys)")
    for (lo, W), wk in zip(wins, selected):
        assert wk.size > W // 4
        A, C = oracle.fill_window(wk, s0, m0, lo, W)
        assert np.array_equal(words[lo // 64:(lo + W) // 64], oracle_windows.pack_bits(A)), lo
        r = oracle.window_ranks(wk, s0, m0, lo, A)
        placed = r != U64MAX
        assert int(placed.sum()) == int(A.sum())
        got = mphf.to_u64(h.lookup(torch.from_numpy(wk[placed].view(np.int64)).cuda()))
        if lo == 0:
            assert np.array_equal(got, r[placed])
        else:
            off = got - r[placed]
            assert np.all(off == off[0]), lo
        # keys that collided in the window go on to deeper levels: their
        # indices are outside the window's range of ranks
        coll = wk[~placed]
        got_c = mphf.to_u64(h.lookup(torch.from_numpy(coll.view(np.int64)).cuda()))
        assert np.all(got_c < N)
    del words

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
    sel_q = torch.randint(0, N, (10**9,), device="cuda",
                          generator=torch.Generator(device="cuda").manual_seed(5))
    q = keys[sel_q]
    del sel_q
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
    # strategy; Sec. 4.5 streams generated keys the same way): equal, bit for bit.
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g2 = mphf.MPHF.build_generated(N, KEY_SEED, 0, gamma=2.0, levels=25, seed=0)
    t1 = time.perf_counter()
    print(f"generated-key build of 1e10 keys: {t1 - t0:.2f} s")
    assert g2.levels() == lv and g2.total_bits == h.total_bits
    assert g2.num_fallback == h.num_fallback
    assert np.array_equal(g2.rank(), h.rank())
    q = keys[::997]
    assert torch.equal(g2.lookup(q), h.lookup(q))
