"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
generator outputs, closed forms, the worked example of Fig. 1, brute force on
tiny inputs, the expectations of Sec. 2.3 / Lemma 1, Table 1, Sec. 3.4 and
Sec. 3.5, and order independence.  A dropped term, a wrong sign or index or a
transposed operand in the oracle fails at least one of them (see the planted
mistakes in ``test_oracle_mutants.py``).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1702_03154_gb300 import inputs

U64 = (1 << 64) - 1


# ---------------------------------------------------------------- hash pieces
def test_mixer_matches_published_splitmix64(golden_dir):
    vals = [int(l, 16) for l in open(os.path.join(golden_dir, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    state = 0
    for v in vals:
        state = (state + 0x9E3779B97F4A7C15) & U64
        assert oracle.mix(state) == v


def test_mixer_is_a_bijection_on_a_sample():
    # Distinct inputs give distinct outputs (the finalizer is invertible).
    xs = inputs.splitmix64_keys(200000, 99)
    ys = np.array([oracle.mix(int(x)) for x in xs[:20000]], dtype=np.uint64)
    assert np.unique(ys).size == ys.size


def test_level_seeds_differ_per_level():
    s = [oracle.level_seed(7, d) for d in range(64)]
    assert len(set(s)) == 64
    assert oracle.level_seed(7, 0) != oracle.level_seed(8, 0)


@pytest.mark.parametrize("h,m,expect", [
    (0, 64, 0),
    (U64, 64, 63),
    (U64, 1 << 40, (1 << 40) - 1),
    (1 << 63, 1000, 500),
    (1 << 62, 64, 16),
    ((1 << 63) - 1, 2, 0),
    (1 << 63, 2, 1),
])
def test_fastrange_closed_forms(h, m, expect):
    assert oracle.fastrange(h, m) == expect


def test_fastrange_against_big_integers():
    rng = np.random.Generator(np.random.PCG64(5))
    for _ in range(2000):
        h = int(rng.integers(0, 1 << 63)) * 2 + int(rng.integers(0, 2))
        m = int(rng.integers(64, 1 << 40))
        assert oracle.fastrange(h, m) == (h * m) >> 64
        assert 0 <= oracle.fastrange(h, m) < m


@pytest.mark.parametrize("n,gamma,expect", [
    (1, 1.0, 64), (64, 1.0, 64), (65, 1.0, 128), (100, 2.0, 256), (1000, 1.5, 1536),
    (10**6, 2.0, 2000000), (10**6 + 1, 2.0, 2000064), (3, 5.0, 64), (13, 5.0, 128),
    (10**8, 1.0, 100000000 + 0 if 10**8 % 64 == 0 else 100000000 + 64 - 10**8 % 64),
])
def test_level_size_rule(n, gamma, expect):
    # |A_d| = gamma |F_d| (Sec. 2.2.4), ceil'd and rounded up to 64-bit words.
    assert oracle.level_bits(n, gamma) == expect
    assert oracle.level_bits(n, gamma) >= gamma * n


# ---------------------------------------------------------- worked example
def test_fig1_worked_example(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "fig1_worked_example.json")))
    names = ["k1", "k2", "k3", "k4", "k5", "k6"]
    key = {nm: 1000 + 17 * i for i, nm in enumerate(names)}
    name = {v: k for k, v in key.items()}
    # Positions consistent with the caption: level 0 places k6 < k3 and makes
    # {k1,k2} and {k4,k5} collide; level 1 places k5 < k1 and makes {k2,k4}
    # collide; level 2 places k2 < k4.
    pos = [
        {"k6": 0, "k3": 1, "k1": 2, "k2": 2, "k4": 4, "k5": 4},
        {"k5": 0, "k1": 1, "k2": 2, "k4": 2},
        {"k2": 0, "k4": 1},
    ]

    def hook(level, k, m):
        return pos[level][name[k]] if level < len(pos) and name[k] in pos[level] else m - 1

    keys = [key[nm] for nm in names]
    h = oracle.build(keys, gamma=g["gamma"], levels=25, seed=0, pos_hook=hook)
    assert h.num_levels == 3
    assert h.level_sizes() == [6, 4, 2, 0]
    out = h.lookup(keys)
    expect = [g["values_1based"][nm] - 1 for nm in names]
    assert out.tolist() == expect
    assert h.key_level(key["k2"]) == g["query_k2_level"]
    assert int(out[1]) + 1 == g["query_k2_value_1based"]
    # A0 holds exactly k3 and k6, A1 k1 and k5, A2 k2 and k4.
    placed = {d: sorted(nm for nm in names if h.key_level(key[nm]) == d) for d in range(3)}
    lv = g["levels_from_caption"]
    assert placed[0] == sorted(lv["A0_placed"])
    assert placed[1] == sorted(lv["A1_placed"])
    assert placed[2] == sorted(lv["A2_placed"])


# ------------------------------------------------------------- brute force
def _is_bijection(out, n):
    return np.array_equal(np.sort(out), np.arange(n, dtype=np.uint64))


@pytest.mark.parametrize("gamma", [1.0, 1.3, 2.0, 5.0])
@pytest.mark.parametrize("levels", [1, 2, 3, 25])
def test_bijection_on_tiny_inputs(gamma, levels):
    for seed in range(60):
        n = 1 + (seed * 37) % 2000
        keys = inputs.splitmix64_keys(n, 1000 + seed)
        h = oracle.build(keys, gamma=gamma, levels=levels, seed=seed)
        out = h.lookup(keys)
        assert _is_bijection(out, n), (gamma, levels, seed, n)
        sizes = h.level_sizes()
        assert sizes[0] == n and sizes[-1] == h.num_fallback
        assert h.num_levels <= levels


def test_brute_force_index_is_rank_of_level_position():
    # Independent characterisation: the index of a placed key is the number of
    # placed keys whose (level offset + position) is smaller; fallback keys come
    # after all placed keys in increasing key order.
    for seed in range(20):
        n = 50 + 31 * seed
        keys = inputs.splitmix64_keys(n, 77 + seed)
        h = oracle.build(keys, gamma=1.0, levels=3, seed=seed)
        lv = h.levels()
        glob = {}
        fb = []
        for x in keys.tolist():
            d = h.key_level(x)
            if d == h.num_levels:
                fb.append(x)
                continue
            n_d, m_d, off_d, s_d = lv[d]
            glob[x] = off_d + oracle.fastrange(oracle.mix(x ^ s_d), m_d)
        order = sorted(glob, key=lambda x: glob[x])
        expect = {x: i for i, x in enumerate(order)}
        for i, x in enumerate(sorted(fb)):
            expect[x] = len(order) + i
        out = h.lookup(keys)
        assert out.tolist() == [expect[x] for x in keys.tolist()]


# --------------------------------------------------------------- statistics
def _build(n, gamma, seed=1, levels=25):
    return oracle.build(inputs.splitmix64_keys(n, seed), gamma=gamma, levels=levels, seed=seed)


@pytest.mark.parametrize("gamma", [1.0, 2.0, 5.0])
def test_placed_fraction_per_level(gamma):
    # Sec. 2.3: a fraction ~ e^{-1/gamma} of F_d is placed at level d; exactly,
    # a key is alone at its position with probability (1 - 1/m_d)^(n_d - 1).
    h = _build(10**6, gamma)
    sizes = h.level_sizes()
    for d in range(4):
        n_d, m_d, _, _ = h.level_info(d)
        if n_d < 2000:
            break
        p = (1.0 - 1.0 / m_d) ** (n_d - 1)
        placed = sizes[d] - sizes[d + 1]
        sigma = math.sqrt(n_d * p * (1 - p))
        assert abs(placed - n_d * p) < 6 * sigma + 1, (d, placed, n_d * p)
        assert abs(p - math.exp(-1.0 / gamma)) < 2e-3


@pytest.mark.parametrize("gamma,expect", [(1.0, math.e), (2.0, 2 * math.exp(0.5)),
                                          (5.0, 5 * math.exp(0.2))])
def test_total_size_matches_gamma_e_1_over_gamma(gamma, expect):
    # Sec. 2.3 / Appendix: sum |A_d| = gamma e^{1/gamma} N.
    h = _build(10**6, gamma)
    assert abs(h.total_bits / 10**6 - expect) / expect < 0.01


def test_bits_per_key_matches_table1(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "table1_bits_per_key.json")))
    for row in g["rows"]:
        h = _build(10**6, row["gamma"], seed=3)
        # minirank (rank_block 1024): one counter per 1024 bits instead of 512
        bpk = h.bits_per_key_sampled(row["rank_block"])
        if row["rank_block"] == 512:
            assert bpk == h.bits_per_key()
        assert abs(bpk - row["bits_per_key"]) <= g["printed_precision"] + 0.01, (row, bpk)
        # the counters of a block size cost exactly 64 / rank_block bits per bit of A
        M = h.total_bits
        want = (M + 64 * math.ceil(M / row["rank_block"]) + 64 * h.num_fallback) / h.N
        assert bpk == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("gamma", [1.0, 2.0, 5.0])
def test_mean_level_is_e_1_over_gamma(gamma):
    # Sec. 4.1: the average number of levels a key visits is e^{1/gamma}.
    h = _build(10**6, gamma)
    visits = sum(h.level_sizes()[:-1]) / 10**6
    assert abs(visits - math.exp(1.0 / gamma)) / math.exp(1.0 / gamma) < 0.01


def test_temporary_set_sizes_match_sec34(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "sec34_temporary_sets.json")))
    for row in g["rows"]:
        h = _build(10**6, row["gamma"], seed=4)
        s = h.level_sizes()
        ratio = (s[1] + s[2]) / s[0]
        assert abs(ratio - row["ratio"]) <= g["printed_precision"] + 0.005, (row, ratio)


@pytest.mark.parametrize("gamma", [1.0, 1.2, 2.0, 5.0])
def test_lemma1_construction_memory(gamma):
    # Lemma 1: m(d) = sum_{i<d} |A_i| + 2|A_d|; max_d m(d)/S <= 1 for
    # gamma <= 1/ln 2, in (1, 2) otherwise, with m(0)/S = 2 e^{-1/gamma}.
    h = _build(10**6, gamma)
    lv = h.levels()
    S = h.total_bits
    m = [sum(x[1] for x in lv[:d]) + 2 * lv[d][1] for d in range(len(lv))]
    R = max(m) / S
    assert abs(m[0] / S - 2 * math.exp(-1 / gamma)) < 0.01
    if gamma <= 1 / math.log(2):
        assert R <= 1.0 + 0.01
    else:
        assert 1.0 < R < 2.0
        assert abs(R - 2 * math.exp(-1 / gamma)) < 0.01


def test_fallback_count_at_gamma1_is_about_1e_5_N():
    # Sec. 3.5: with D = 25 levels, about 1e-5 N keys reach the hash table at
    # gamma = 1 (q^25 N with q = 1 - 1/e) and practically none at gamma >= 2.
    n = 4 * 10**6
    h = _build(n, 1.0, seed=11)
    expect = (1 - math.exp(-1)) ** 25 * n
    assert abs(expect / n - 1e-5) < 0.1e-5
    assert abs(h.num_fallback - expect) < 6 * math.sqrt(expect)
    assert _build(10**6, 2.0, seed=11).num_fallback == 0


# --------------------------------------------------------------- invariants
@pytest.mark.parametrize("gamma,levels", [(1.0, 25), (2.0, 25), (1.0, 4)])
def test_structural_invariants(gamma, levels):
    n = 200000
    h = _build(n, gamma, seed=21, levels=levels)
    sizes = h.level_sizes()
    A = h.bits()
    total = 0
    for d in range(h.num_levels):
        a = h.level_bits_words(d)
        c = h.collision_bits(d)
        assert not np.any(a & c)                             # Alg. 2 footnote
        w = int(np.unpackbits(a.view(np.uint8)).sum())
        assert w == sizes[d] - sizes[d + 1]                  # weight(A_d)
        total += w
    assert total + h.num_fallback == n
    bitsA = np.unpackbits(A.view(np.uint8), bitorder="little").astype(np.int64)
    ones = np.concatenate([[0], np.cumsum(bitsA)])
    rank = h.rank()
    assert rank.size == (h.total_bits + 511) // 512
    assert np.array_equal(rank, ones[np.arange(rank.size) * 512].astype(np.uint64))
    fb = h.fallback()
    assert np.all(fb[1:] > fb[:-1])


def test_order_independence():
    keys = inputs.splitmix64_keys(300000, 31)
    a = oracle.build(keys, gamma=1.0, levels=25, seed=5)
    b = oracle.build(inputs.shuffled(keys, 9), gamma=1.0, levels=25, seed=5)
    assert a.levels() == b.levels()
    assert np.array_equal(a.bits(), b.bits())
    assert np.array_equal(a.rank(), b.rank())
    assert np.array_equal(a.fallback(), b.fallback())
    assert np.array_equal(a.lookup(keys), b.lookup(keys))


# --------------------------------------------------------------- edge cases
def test_empty_and_single_key():
    h = oracle.build(np.zeros(0, dtype=np.uint64), 2.0, 25, 0)
    assert h.num_levels == 0 and h.total_bits == 0 and h.num_fallback == 0
    assert h.lookup([1, 2, 3]).tolist() == [U64] * 3
    h1 = oracle.build([12345], 2.0, 25, 0)
    assert h1.lookup([12345]).tolist() == [0]
    assert h1.num_levels == 1 and h1.total_bits == 64


def test_duplicates_are_reported():
    keys = inputs.splitmix64_keys(1000, 3)
    keys[500] = keys[17]
    with pytest.raises(oracle.OracleError) as e:
        oracle.build(keys, 2.0, 25, 0)
    assert e.value.code == oracle.EDUPLICATE
    with pytest.raises(oracle.OracleError):
        oracle.build(np.array([5, 5], dtype=np.uint64), 1.0, 3, 0)


@pytest.mark.parametrize("gamma,levels", [(0.5, 25), (float("nan"), 25), (float("inf"), 25),
                                          (2.0, 0), (2.0, 65)])
def test_invalid_arguments(gamma, levels):
    with pytest.raises(oracle.OracleError) as e:
        oracle.build([1, 2, 3], gamma, levels, 0)
    assert e.value.code == oracle.EINVAL


def test_single_level_sends_colliders_to_fallback():
    keys = inputs.splitmix64_keys(5000, 8)
    h = oracle.build(keys, gamma=1.0, levels=1, seed=2)
    n_fb = h.num_fallback
    assert n_fb > 0
    out = h.lookup(keys)
    assert _is_bijection(out, keys.size)
    fb = h.fallback()
    pos = {int(x): i for i, x in enumerate(fb)}
    for x, v in zip(keys.tolist(), out.tolist()):
        if x in pos:
            assert v == keys.size - n_fb + pos[x]


def test_non_member_keys_follow_algorithm3():
    keys = inputs.splitmix64_keys(20000, 12)
    h = oracle.build(keys, gamma=1.0, levels=2, seed=4)
    others = inputs.splitmix64_keys(20000, 13)
    out = h.lookup(others)
    ok = (out < keys.size) | (out == np.uint64(U64))
    assert np.all(ok)
    assert np.any(out == np.uint64(U64))       # some fall through every level
    assert np.array_equal(out, h.lookup(others))


# ---------------------------------------------------------------- string keys
# Strings become 64-bit keys before the method runs (Sec. 4.4).  The pins tie
# the conversion to the published SplitMix64 outputs: the first state of a
# string of length len is output len of the generator, and a group equal to
# that state cancels it (mix(0) = 0), so chosen strings have keys that are
# themselves generator outputs.
def test_empty_string_key_is_generator_output_0(golden_dir):
    first = int([l for l in open(os.path.join(golden_dir, "splitmix64_seed0.txt"))
                 if l.strip() and not l.startswith("#")][0], 16)
    assert oracle.string_key(b"", 0) == first
    for seed in (1, 77, 2**63 + 5):
        assert oracle.string_key(b"", seed) == int(inputs.splitmix64_keys(1, seed)[0])


def test_string_key_group_cancels_the_length_state():
    # A string of 8 bytes whose value (little-endian) is the first state
    # mix(seed + 9 G) = generator output 8 has key mix(0) = 0.
    for seed in (0, 3, 991):
        state = int(inputs.splitmix64_keys(9, seed)[8])
        assert oracle.string_key(state.to_bytes(8, "little"), seed) == 0
        assert oracle.string_key(state.to_bytes(8, "big"), seed) != 0


def test_string_key_groups_chain_in_order():
    # 16 bytes: group 0 cancels the first state (output 16 of the generator),
    # so the key is mix(group 1); with group 1 = t + (j + 1) G that is output j
    # of a generator started at t.
    G = 0x9E3779B97F4A7C15
    for seed, t, j in ((0, 5, 0), (12, 99, 7), (2**40, 1, 3)):
        first = int(inputs.splitmix64_keys(17, seed)[16])
        g1 = (t + (j + 1) * G) & U64
        s = first.to_bytes(8, "little") + g1.to_bytes(8, "little")
        assert oracle.string_key(s, seed) == int(inputs.splitmix64_keys(j + 1, t)[j])
        # swapping the two groups breaks it
        assert oracle.string_key(s[8:] + s[:8], seed) != int(inputs.splitmix64_keys(j + 1, t)[j])


def test_string_keys_distinct_in_the_last_group():
    # For fixed length and leading groups the key is a bijection of the last
    # group: distinct last groups can never collide.
    prefix = b"0123456789abcdef"
    tails = inputs.splitmix64_keys(20000, 5)
    data = np.frombuffer(b"".join(prefix + int(t).to_bytes(8, "little") for t in tails),
                         dtype=np.uint8)
    off = np.arange(0, 24 * (tails.size + 1), 24, dtype=np.uint64)
    k = oracle.string_keys(data, off, 9)
    assert np.unique(k).size == tails.size


def test_string_key_depends_on_length_and_seed():
    data, off = inputs.random_words(2000, 3, length=0, max_length=30)
    for i in range(0, 2000, 7):
        s = data[int(off[i]):int(off[i + 1])].tobytes()
        assert oracle.string_key(s, 1) != oracle.string_key(s + b"\0", 1)
        assert oracle.string_key(s, 1) != oracle.string_key(s, 2)


def test_string_key_batch_matches_single():
    data, off = inputs.random_words(3000, 4, length=1, max_length=40)
    k = oracle.string_keys(data, off, 123)
    for i in range(0, 3000, 11):
        assert int(k[i]) == oracle.string_key(data[int(off[i]):int(off[i + 1])].tobytes(), 123)


def test_string_keys_bits_per_key_matches_table2(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "table2_string_keys.json")))
    data, off = inputs.random_words(200000, 6, length=18)
    keys = oracle.string_keys(data, off, 0)
    assert np.unique(keys).size == keys.size
    o = oracle.build(keys, gamma=g["gamma"], levels=25, seed=0)
    assert abs(o.bits_per_key() - g["bits_per_key"]) <= g["printed_precision"]


# ------------------------------------------------- multi-rank level exchange
# A monolithic multi-GPU level (keys of F_d sharded over ranks) needs each
# rank's ArrayFill of its shard and one exchange that merges them.  The merge
# is pinned to brute force (count the keys per position) and to the level
# arrays of a whole build.
def _brute_fill(keys, s_d, m):
    pos = np.array([oracle.fastrange(oracle.mix(int(k) ^ s_d), m) for k in keys], dtype=np.int64)
    cnt = np.bincount(pos, minlength=m)
    return (cnt == 1).astype(np.uint8), (cnt >= 2).astype(np.uint8)


def test_level_fill_is_brute_force_counting():
    keys = inputs.splitmix64_keys(3000, 140)
    for m in (64, 2048, 6000):
        s = oracle.level_seed(5, 2)
        A, C = oracle.fill_level(keys, s, m)
        bA, bC = _brute_fill(keys, s, m)
        assert np.array_equal(A, bA) and np.array_equal(C, bC)


@pytest.mark.parametrize("K", [2, 3, 4, 7])
def test_sharded_fills_merge_to_the_whole_fill(K):
    keys = inputs.splitmix64_keys(5000, 141)
    s, m = oracle.level_seed(1, 0), 4096  # crowded: many collisions of every kind
    A, C = oracle.fill_level(keys, s, m)
    rng = np.random.default_rng(K)
    owner = rng.integers(0, K, size=keys.size)
    parts = [oracle.fill_level(keys[owner == r], s, m) for r in range(K)]
    mA, mC = parts[0]
    for a, c in parts[1:]:
        mA, mC = oracle.merge_fill(mA, mC, a, c)
    assert np.array_equal(mA, A) and np.array_equal(mC, C)
    # any merge order gives the same result (commutative, associative)
    rA, rC = parts[-1]
    for a, c in reversed(parts[:-1]):
        rA, rC = oracle.merge_fill(a, c, rA, rC)
    assert np.array_equal(rA, A) and np.array_equal(rC, C)
    # the empty fill is the identity
    z = np.zeros(m, dtype=np.uint8)
    eA, eC = oracle.merge_fill(A, C, z, z)
    assert np.array_equal(eA, A) and np.array_equal(eC, C)


def test_sharded_level0_equals_the_builds_A0():
    keys = inputs.splitmix64_keys(20000, 142)
    o = oracle.build(keys, gamma=2.0, levels=25, seed=9)
    n0, m0, off0, s0 = o.level_info(0)
    half = keys.size // 2
    A, C = oracle.merge_fill(*oracle.fill_level(keys[:half], s0, m0),
                             *oracle.fill_level(keys[half:], s0, m0))
    words = o.level_bits_words(0)
    bits = np.unpackbits(words.view(np.uint8), bitorder="little")[:m0]
    assert np.array_equal(A, bits)
    assert int(A.sum()) == n0 - o.level_info(1)[0]


# --------------------------------------------------- one window of a level
# A check of a level too large for the oracle to build whole (1e10 keys)
# fills one window of its positions from the keys hashed into it.  Pinned to
# brute-force counting and to the level arrays of a whole build.
@pytest.mark.parametrize("m,lo,W", [(6000, 0, 6000), (6000, 64, 1024), (6000, 5999, 1),
                                    (6000, 4000, 2000), (2048, 100, 37)])
def test_window_fill_is_brute_force_counting(m, lo, W):
    keys = inputs.splitmix64_keys(3000, 143)
    s = oracle.level_seed(7, 0)
    bA, bC = _brute_fill(keys, s, m)
    A, C = oracle.fill_window(keys, s, m, lo, W)
    assert np.array_equal(A, bA[lo:lo + W]) and np.array_equal(C, bC[lo:lo + W])
    sel = oracle.select_window(keys, s, m, lo, W)
    pos = np.array([oracle.fastrange(oracle.mix(int(k) ^ s), m) for k in keys])
    assert np.array_equal(sel, keys[(pos >= lo) & (pos < lo + W)])
    # the selected keys alone give the same window
    A2, C2 = oracle.fill_window(sel, s, m, lo, W)
    assert np.array_equal(A2, A) and np.array_equal(C2, C)


def test_window_of_level0_equals_the_builds_A0():
    keys = inputs.splitmix64_keys(30000, 144)
    o = oracle.build(keys, gamma=2.0, levels=25, seed=10)
    n0, m0, off0, s0 = o.level_info(0)
    bits = np.unpackbits(o.level_bits_words(0).view(np.uint8), bitorder="little")[:m0]
    for lo, W in ((0, 640), (1280, 4096), (m0 - 512, 512)):
        A, _ = oracle.fill_window(oracle.select_window(keys, s0, m0, lo, W), s0, m0, lo, W)
        assert np.array_equal(A, bits[lo:lo + W])


def test_window_ranks_of_the_first_window_are_level0_indices():
    # For the window at the start of A the rank inside the window is the
    # index itself: equal to Algorithm 3's answer for every key placed there.
    keys = inputs.splitmix64_keys(30000, 145)
    o = oracle.build(keys, gamma=2.0, levels=25, seed=11)
    n0, m0, off0, s0 = o.level_info(0)
    lvl = np.array([o.key_level(int(k)) for k in keys])
    for W in (m0, 4096, 64):
        A, _ = oracle.fill_window(keys, s0, m0, 0, W)
        r = oracle.window_ranks(keys, s0, m0, 0, A)
        pos = np.array([oracle.fastrange(oracle.mix(int(k) ^ s0), m0) for k in keys])
        placed = (lvl == 0) & (pos < W)
        assert np.array_equal(r[placed], o.lookup(keys[placed]))
        assert np.all(r[~placed] == np.uint64((1 << 64) - 1))
    # a later window: ranks are the indices minus the ones before the window
    lo, W = 2048, 4096
    A, _ = oracle.fill_window(keys, s0, m0, lo, W)
    r = oracle.window_ranks(keys, s0, m0, lo, A)
    pos = np.array([oracle.fastrange(oracle.mix(int(k) ^ s0), m0) for k in keys])
    placed = (lvl == 0) & (pos >= lo) & (pos < lo + W)
    base = int(o.rank()[lo // 512])
    assert np.array_equal(r[placed] + np.uint64(base), o.lookup(keys[placed]))


def test_window_selection_over_processes_equals_one_pass():
    # the helper of the 1e10-key check splits the key stream over spawned
    # processes; the union of their selections is the single-pass selection
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import oracle_windows
    n, s, m = 300007, oracle.level_seed(0, 0), oracle.level_bits(300007, 2.0)
    wins = [(0, 4096), (m // 2 // 64 * 64, 8192), (m - 640, 640)]
    got = oracle_windows.finish_selection(
        oracle_windows.start_selection(n, 4, s, m, wins, workers=3))
    keys = inputs.splitmix64_keys(n, 4)
    for (lo, W), g in zip(wins, got):
        assert np.array_equal(g, oracle.select_window(keys, s, m, lo, W))
    A, _ = oracle.fill_window(keys, s, m, 0, 4096)
    assert np.array_equal(np.unpackbits(oracle_windows.pack_bits(A).view(np.uint8),
                                        bitorder="little"), A)


# ------------------------------------------------------ partitioned mode
# K independent functions over a hash split of the keys (the partitioning
# Sec. 4.3 calls applicable to this method): pinned to the plain build at
# K = 1, to brute-force bijection, to the per-part index ranges, to the
# power-of-two closed form of the split, and to the multinomial part sizes.
def test_one_part_is_the_plain_build():
    keys = inputs.splitmix64_keys(20011, 150)
    o = oracle.build(keys, gamma=2.0, levels=25, seed=3)
    P = oracle.PartitionedOracle(keys, 1, 77, gamma=2.0, levels=25, seed=3)
    assert np.array_equal(P.lookup(keys), o.lookup(keys))
    assert P.functions[0].levels() == o.levels()


@pytest.mark.parametrize("K,n", [(2, 1000), (3, 5003), (7, 777), (16, 20000), (64, 3000)])
def test_partitioned_indices_are_a_bijection(K, n):
    keys = inputs.splitmix64_keys(n, 151 + K)
    P = oracle.PartitionedOracle(keys, K, 5, gamma=1.0, levels=3, seed=1)
    out = P.lookup(keys)
    assert np.array_equal(np.sort(out), np.arange(n, dtype=np.uint64))
    p = oracle.parts(keys, K, 5)
    sizes = np.bincount(p.astype(np.int64), minlength=K)
    assert sizes.sum() == n
    assert np.array_equal(P.offsets[1:] - P.offsets[:-1], sizes.astype(np.uint64))
    for k in range(K):   # each key's index lies in its part's range
        sel = p == k
        assert np.all((out[sel] >= P.offsets[k]) & (out[sel] < P.offsets[k + 1]))
        # and is its part's own function's index, shifted
        assert np.array_equal(out[sel] - P.offsets[k], P.functions[k].lookup(keys[sel]))
    # non-members: either a miss or some index of the part they hash to
    other = inputs.splitmix64_keys(3000, 152)
    r = P.lookup(other)
    po = oracle.parts(other, K, 5)
    hit = r != np.uint64((1 << 64) - 1)
    assert np.all((r[hit] >= P.offsets[po[hit]]) & (r[hit] < P.offsets[po[hit] + 1]))


def test_part_split_closed_form_for_powers_of_two():
    # with K = 2^j the part is the top j bits of the part hash
    xs = inputs.splitmix64_keys(2000, 153)
    s = oracle.mix(9)
    for j in (1, 3, 10):
        for x in xs[:200]:
            h = oracle.mix(int(x) ^ s)
            assert oracle.part_of(int(x), 1 << j, 9) == h >> (64 - j)
    # and the split is close to uniform (multinomial, 6 sigma per part)
    K, n = 10, 200000
    c = np.bincount(oracle.parts(inputs.splitmix64_keys(n, 154), K, 9).astype(np.int64),
                    minlength=K)
    sd = np.sqrt(n * (1 / K) * (1 - 1 / K))
    assert np.all(np.abs(c - n / K) < 6 * sd)
