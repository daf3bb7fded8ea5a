"""String keys on the GPU (Sec. 4.4, Table 2) against the oracle, bit for bit.

The device conversion of byte strings to 64-bit keys must equal the oracle's
for every string: lengths 0 to 40 bytes, strings starting at every byte
alignment, a buffer whose last string ends at an odd byte.  A function built
over the keys of random 18-character words must equal the oracle's build on
the same keys, give each word its index, and have Table 2's 3.7 bits/key.
Offsets outside the buffer are refused without a read.
"""
import json
import os

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


@pytest.mark.parametrize("n,lo,hi,seed", [(1, 0, 0, 0), (5000, 0, 40, 1), (100003, 18, 18, 2),
                                          (77777, 1, 9, 2**63 + 11)])
def test_string_keys_match_oracle(M, n, lo, hi, seed):
    data, off = inputs.random_words(n, 80 + n, length=lo, max_length=hi)
    want = oracle.string_keys(data, off, seed)
    got = M.to_u64(M.string_keys(data, off, seed))
    assert np.array_equal(got, want)


def test_every_alignment_and_ragged_end(M):
    # the same words placed at byte offsets 0..15 of the device buffer
    data, off = inputs.random_words(3001, 90, length=0, max_length=33)
    want = oracle.string_keys(data, off, 5)
    for shift in range(16):
        buf = torch.zeros(data.size + shift, dtype=torch.uint8, device="cuda")
        buf[shift:] = torch.from_numpy(data).cuda()
        got = M.to_u64(M.string_keys(buf, off + np.uint64(shift), 5))
        assert np.array_equal(got, want), shift


def test_string_function_matches_oracle_and_table2(M, golden_dir):
    g = json.load(open(os.path.join(golden_dir, "table2_string_keys.json")))
    data, off = inputs.random_words(10**6, 91, length=18)
    keys = oracle.string_keys(data, off, 0)
    o = oracle.build(keys, gamma=g["gamma"], levels=25, seed=0)
    dk = M.string_keys(data, off, 0)
    assert np.array_equal(M.to_u64(dk), keys)
    h = M.MPHF.build(dk, gamma=g["gamma"], levels=25, seed=0)
    assert h.levels() == o.levels()
    assert np.array_equal(h.bits(), o.bits())
    idx = M.to_u64(h.lookup(dk))
    assert np.array_equal(idx, o.lookup(keys))
    assert np.array_equal(np.sort(idx), np.arange(keys.size, dtype=np.uint64))
    assert abs(h.bits_per_key() - g["bits_per_key"]) <= g["printed_precision"]


@pytest.mark.parametrize("bad", ["past_end", "decreasing"])
def test_bad_offsets_are_refused(M, bad):
    data, off = inputs.random_words(100, 92, length=5, max_length=12)
    off = off.copy()
    if bad == "past_end":
        off[-1] = np.uint64(data.size + 1)
    else:
        off[50], off[51] = off[51], off[50]
    with pytest.raises(M.MPHFError) as e:
        M.string_keys(data, off, 0)
    assert e.value.code == M.EINVAL
