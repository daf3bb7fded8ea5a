"""Planted mistakes in the oracle must fail its pins.

Each case compiles a copy of ``oracle/mphf_oracle.c`` with one plausible
mistake (a dropped term, a wrong index or comparison, a transposed branch)
on the CPU, runs the pin suite against it in a subprocess and expects a
failure.  This shows the pins in ``test_oracle_pins.py`` constrain every step
of the oracle, not just its output format.
"""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mphf_oracle.c")

MUTANTS = {
    # ArrayFill: a third key at a collided position sets A again.
    "fill_ignores_C": ("if (A[p] == 0 && C[p] == 0) {", "if (A[p] == 0) {"),
    # ArrayFill: a collision leaves A set.
    "collision_keeps_A": ("A[p] = 0;\n        C[p] = 1;", "C[p] = 1;"),
    # Alg. 1: the colliding keys are dropped and the placed ones kept.
    "compaction_inverted": ("if (A[p] == 0)\n                Fnext[nn++] = F[k];",
                            "if (A[p] == 1)\n                Fnext[nn++] = F[k];"),
    # Sec. 2.2.3: inclusive rank.
    "rank_inclusive": ("for (uint64_t t = b * ORACLE_RANK_BLOCK; t < g; t++)",
                       "for (uint64_t t = b * ORACLE_RANK_BLOCK; t <= g; t++)"),
    # Sec. 3.1: checkpoint taken after the block's first bit.
    "checkpoint_late": ("if (g % ORACLE_RANK_BLOCK == 0)\n            h->rank[g / ORACLE_RANK_BLOCK] = ones;\n        ones += h->bitA[g];",
                        "ones += h->bitA[g];\n        if (g % ORACLE_RANK_BLOCK == 0)\n            h->rank[g / ORACLE_RANK_BLOCK] = ones;"),
    # Sec. 2.1: the same hash function at every level.
    "level_seed_ignores_d": ("return oracle_mix(oracle_mix(seed) + (uint64_t)d);",
                             "return oracle_mix(oracle_mix(seed) + 0 * (uint64_t)d);"),
    # Sec. 2.2.4: gamma dropped from |A_d|.
    "size_ignores_gamma": ("double t = gamma * (double)n;", "double t = (double)n;"),
    # Sec. 3.5 / Alg. 1 footnote: fallback indices shifted by one.
    "fallback_offset": ("return h->N - h->n_fb + lo;", "return h->N - h->n_fb + lo + 1;"),
    # Mixer: one constant mistyped.
    "mixer_constant": ("0x94D049BB133111EBULL", "0x94D049BB133111EDULL"),
    # Reduction: shift of 63 instead of 64.
    "fastrange_shift": ("(unsigned __int128)m) >> 64);", "(unsigned __int128)m) >> 63);"),
    # Offsets: each level starts at bit 0.
    "offset_not_accumulated": ("off += h->m[i];", "off += 0 * h->m[i];"),
    # Sec. 4.3 minirank: the counter interval ignored (always 512).
    "rank_sampling_ignored": ("uint64_t counters = (h->M + rank_block - 1) / rank_block;",
                              "uint64_t counters = (h->M + 511) / 512;"),
    # Multi-rank merge: two single hits on different ranks not seen as a collision.
    "merge_drops_cross_collision": ("(unsigned char)(C1[p] | C2[p] | (A1[p] & A2[p]))",
                                    "(unsigned char)(C1[p] | C2[p])"),
    # Multi-rank merge: a collided position keeps its A bit.
    "merge_keeps_collided_A": ("A1[p] = (unsigned char)((A1[p] | A2[p]) & !c);",
                               "A1[p] = (unsigned char)(A1[p] | A2[p]);"),
    # String keys (Sec. 4.4): the length left out of the first state.
    "string_length_dropped": ("oracle_mix(seed + (len + 1) * 0x9E3779B97F4A7C15ULL)",
                              "oracle_mix(seed + 1 * 0x9E3779B97F4A7C15ULL)"),
    # String keys: groups read big-endian.
    "string_big_endian": ("w |= byte << (8 * i);", "w |= byte << (8 * (7 - i));"),
    # Partitioned mode: the part hash keyed by the raw seed.
    "part_seed_unmixed": ("oracle_mix(x ^ oracle_mix(part_seed))", "oracle_mix(x ^ part_seed)"),
    # Partitioned mode: the split reduced onto K - 1 parts.
    "part_range_short": ("(uint64_t)K);\n}", "(uint64_t)K - 1);\n}"),
    # String keys: a group OR-ed into the state instead of XOR-ed.
    "string_group_or": ("h = oracle_mix(h ^ w);", "h = oracle_mix(h | w);"),
}


def _compile(tag, old, new, tmp):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutant {tag}: anchor not found exactly once"
    path_c = os.path.join(tmp, f"{tag}.c")
    open(path_c, "w").write(src.replace(old, new))
    path_so = os.path.join(tmp, f"lib{tag}.so")
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-shared", "-fPIC",
                           "-o", path_so, path_c, "-lm"])
    return path_so


@pytest.mark.parametrize("tag", sorted(MUTANTS))
def test_planted_mistake_is_caught(tag):
    old, new = MUTANTS[tag]
    with tempfile.TemporaryDirectory() as tmp:
        so = _compile(tag, old, new, tmp)
        env = dict(os.environ, MPHF_ORACLE_LIB=so)
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode != 0, f"mutant {tag} passed every pin:\n{r.stdout[-2000:]}"
