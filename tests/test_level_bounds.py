"""The bucketed build's level-1 arena bound, checked on the host (no GPU).

A bucketed build allocates level 1's bucket arena before level 0 runs, from
a bound n1_hi on |F_1| (keys not alone at level 0: mean N - N (1 - 1/m_0)^(N-1),
Sec. 2.3, standard deviation below sqrt(N)).  Whatever size the device then
picks for |F_1| = n <= n1_hi keys (B buckets of P positions, cap slots each)
must fit: B cap <= capY and B <= Bb.  The library's own sizing routine and
bound are called here through host-only test hooks, over sizes around every
bucket-width switch, and n1_hi is compared with the oracle's |F_1|.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1702_03154_gb300 import inputs


@pytest.fixture(scope="module")
def M():
    from paper_1702_03154_gb300 import build_ext, mphf
    build_ext.build()
    return mphf


def level_bits(n, gamma):
    return max(64, ((math.ceil(gamma * n) + 63) // 64) * 64)


def probe_sizes(n1_hi, gamma, btarget, rng):
    ns = {1, 2, 63, 64, 65, 1000, n1_hi, max(1, n1_hi - 1), n1_hi // 2 + 1}
    ns |= {int(x) for x in rng.integers(1, n1_hi + 1, 400)}
    # around each switch of the bucket width: m_d / btarget crossing 2^k
    for k in range(12, 19):
        edge = (2 ** k) * btarget / gamma
        for dn in range(-3, 4):
            v = int(edge) + dn
            if 1 <= v <= n1_hi:
                ns.add(v)
    return sorted(ns)


@pytest.mark.parametrize("gamma", [1.0, 1.3, 2.0, 5.0, 10.0])
@pytest.mark.parametrize("btarget", [456, 608, 1216])
@pytest.mark.parametrize("N", [20000, 123457, 10**6, 10**7, 10**8, 2 * 10**8])
def test_level1_arena_bound_covers_every_level_size(M, gamma, btarget, N):
    rng = np.random.default_rng(N + btarget)
    n1_hi, capY, Bb = M.debug_level1_bound(N, gamma, btarget)
    m0 = level_bits(N, gamma)
    mean = N - N * (1.0 - 1.0 / m0) ** (N - 1)
    assert n1_hi >= min(N, mean + 10 * math.sqrt(N))
    for n in probe_sizes(n1_hi, gamma, btarget, rng):
        B, cap, P = M.debug_size_level(n, gamma, btarget)
        assert P & (P - 1) == 0 and 4096 <= P <= 262144
        assert B * P >= level_bits(n, gamma)
        assert B <= Bb, (n, B, Bb)
        assert B * cap <= capY, (n, B, cap, capY)


@pytest.mark.parametrize("gamma", [1.0, 2.0, 5.0])
def test_level1_bound_holds_for_the_oracles_level_1(M, gamma):
    # the oracle's |F_1| on a real key set lies inside the bound (far inside:
    # ten standard deviations)
    N = 300000
    keys = inputs.splitmix64_keys(N, 62)
    o = oracle.build(keys, gamma=gamma, levels=2, seed=0)
    n1 = o.level_sizes()[1]
    n1_hi, _, _ = M.debug_level1_bound(N, gamma, 608)
    assert n1 <= n1_hi
    assert n1_hi - n1 > 5 * math.sqrt(N)
