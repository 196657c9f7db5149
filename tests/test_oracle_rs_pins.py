"""Pins of the oracle's splitting process (Rao-Sandelius with a Fisher-Yates cutoff B; the
introduction's passage on splitting processes and Table 1's third row) against what the
mathematics fixes, not against the oracle itself:
  * exact uniformity: an exhaustive walk of every bit and draw, cut at a number of split levels,
    gives every permutation the same probability mass (the ordered partition into segments is
    exchangeable); a Sattolo-style off-by-one in the Fisher-Yates range breaks it;
  * the expected number of split bits equals the exact recursion for a trie with cutoff B;
  * n <= B reduces to a textbook Fisher-Yates on the RS_LEAF stream of segment 0;
  * n = 2, B = 1 worked by hand: the first level whose two bits differ decides the order;
  * outputs are permutations, and a shuffle is the input gathered by the perm (data-oblivious).
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("n,B,levels", [(2, 1, 6), (3, 1, 5), (4, 1, 4), (4, 2, 4), (5, 2, 3),
                                        (5, 1, 3), (6, 3, 3), (6, 2, 2)])
def test_splitting_process_is_exactly_uniform_on_finished_paths(n, B, levels):
    num, den, paths, unres = oracle.enumerate_rs(n, B, levels)
    assert len(num) == math.factorial(n)
    assert len(set(num)) == 1, "permutations reached with different probabilities"
    assert sum(num) + unres == den  # the walk covers the whole probability space
    assert sum(num) > 0


def test_planted_fisher_yates_range_breaks_uniformity():
    num, den, _, _ = oracle.enumerate_rs(4, 3, 4, mode=oracle.PLANT_FY_RANGE)
    assert len(set(num)) > 1


def test_unfinished_mass_matches_the_no_split_probability():
    """n = 2, B = 1: a level leaves the pair unsplit iff its two bits agree (probability 1/2),
    so the mass cut off after L levels is exactly 2^-L."""
    for L in range(1, 7):
        num, den, _, unres = oracle.enumerate_rs(2, 1, L)
        assert Fraction(unres, den) == Fraction(1, 2 ** L)
        assert Fraction(num[0], den) == Fraction(num[1], den) == (1 - Fraction(1, 2 ** L)) / 2


def _expected_split_bits(n: int, B: int) -> float:
    """E[bits drawn by the splits] for a segment of m elements: 0 if m <= B, else
    m + sum_k C(m,k) 2^-m (E(k) + E(m-k)), solved for E(m) (the k = 0, m terms hold E(m))."""
    E = [0.0] * (n + 1)
    for m in range(B + 1, n + 1):
        acc = float(m)
        for k in range(1, m):
            acc += math.comb(m, k) / 2.0 ** m * (E[k] + E[m - k])
        E[m] = acc / (1.0 - 2.0 / 2.0 ** m)
    return E[n]


def test_mean_split_bits_match_the_trie_recursion():
    n, B, trials = 300, 8, 400
    want = _expected_split_bits(n, B)
    got = np.array([oracle.rs_perm(n, s, B)[1].coin_bits for s in range(1, trials + 1)],
                   dtype=np.float64)
    se = got.std(ddof=1) / math.sqrt(trials)
    assert abs(got.mean() - want) < 4 * se, (got.mean(), want, se)


def test_n_at_most_B_is_a_textbook_fisher_yates_on_segment_zero():
    n, B, seed = 200, 256, 11
    a = list(range(n))
    for i in range(n - 1, 0, -1):
        j, _ = oracle.draw(seed, oracle.TAG_RS_LEAF, 0, 0, i, i + 1)
        a[i], a[j] = a[j], a[i]
    got, st = oracle.rs_perm(n, seed, B)
    assert got.tolist() == a
    assert st.coin_bits == 0 and st.merges == 0


def _rs_bit(seed: int, level: int, p: int) -> int:
    w = oracle.philox([p >> 7, 0, (oracle.TAG_RS_COIN << 16) | level, 0],
                      [seed & 0xFFFFFFFF, seed >> 32])
    return int((int(w[(p >> 5) & 3]) >> (p & 31)) & 1)


def test_pair_with_cutoff_one_worked_by_hand():
    for seed in range(1, 200):
        level = 0
        while _rs_bit(seed, level, 0) == _rs_bit(seed, level, 1):
            level += 1
        want = [0, 1] if _rs_bit(seed, level, 0) == 0 else [1, 0]
        got, st = oracle.rs_perm(2, seed, 1)
        assert got.tolist() == want, seed
        assert st.levels == level + 1 and st.coin_bits == 2 * (level + 1)


@pytest.mark.parametrize("n,B", [(1, 1), (7, 1), (1000, 3), (4097, 64), (100_003, 512)])
def test_outputs_are_permutations_and_shuffles_are_data_oblivious(n, B):
    p, _ = oracle.rs_perm(n, 5, B)
    assert np.array_equal(np.sort(p), np.arange(n, dtype=np.uint32))
    rec = np.stack([np.arange(n, dtype=np.uint32) * 3 + 1, np.arange(n, dtype=np.uint32)], 1)
    got, _ = oracle.rs_shuffle(rec, 5, B)
    assert np.array_equal(got, rec[p])
