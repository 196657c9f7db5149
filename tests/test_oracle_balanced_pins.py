"""Pins of the oracle's balanced-word merge (mode BALANCED; the idea of Section 3: a uniform word
in C(n1 + n2, n1) interleaving two uniformly shuffled halves gives a uniform permutation, by the
bijection lemma of Section 3.2). The word is the labels of the two halves merged by the merge's own
coin loop and random insertions; the data is then interleaved stably by it.
  * exact uniformity by enumeration: every permutation of n <= 6, every cutoff, probability 1/n!;
  * one merge: the first half's position set is uniform over C(a + b, a);
  * a planted off-by-one in the insertion range breaks it;
  * each half keeps its order in the merged output (no insertion moves an element);
  * the coins, break steps and draws are the stable merge's: the same random bits."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_balanced_merge_shuffle_is_exactly_uniform(n):
    for B in range(1, n + 1):
        num, den, _ = oracle.enumerate_perm(n, B, oracle.BALANCED)
        assert len(set(num)) == 1 and sum(num) == den, (n, B)


@pytest.mark.parametrize("a,b", [(1, 1), (2, 3), (4, 4), (5, 2), (3, 6)])
def test_balanced_word_is_uniform_over_position_sets(a, b):
    num, den, _ = oracle.enumerate_merge(a, b, oracle.BALANCED)
    nz = [x for x in num if x]
    assert len(nz) == math.comb(a + b, a) and len(set(nz)) == 1
    assert sum(nz) == den


def test_planted_insertion_range_breaks_uniformity():
    num, _, _ = oracle.enumerate_merge(4, 2, oracle.BALANCED | oracle.PLANT_TAIL_RANGE)
    nz = [x for x in num if x]
    assert len(set(nz)) > 1
    num, _, _ = oracle.enumerate_perm(5, 1, oracle.BALANCED | oracle.PLANT_TAIL_RANGE)
    assert len(set(num)) > 1
    num, _, _ = oracle.enumerate_perm(5, 1, oracle.BALANCED | oracle.PLANT_NO_TAIL)
    assert len(set(num)) > 1


def test_halves_keep_their_order_and_bits_match_the_stable_merge():
    rng = np.random.default_rng(3)
    for trial in range(50):
        n1, n2 = int(rng.integers(1, 300)), int(rng.integers(1, 300))
        vals = np.arange(n1 + n2, dtype=np.uint32)
        out, T, st = oracle.merge(vals, n1, 100 + trial, mode=oracle.BALANCED)
        _, T0, st0 = oracle.merge(vals, n1, 100 + trial)
        first = out[out < n1]
        second = out[out >= n1]
        assert np.array_equal(first, np.arange(n1)) and np.array_equal(second, np.arange(n1, n1 + n2))
        assert T == T0 and st.total_bits == st0.total_bits


@pytest.mark.parametrize("n,B", [(1000, 16), (100_003, 256)])
def test_balanced_perm_is_a_permutation_and_data_oblivious(n, B):
    p, st = oracle.perm(n, 4, B, oracle.BALANCED)
    assert np.array_equal(np.sort(p), np.arange(n, dtype=np.uint32))
    q, _ = oracle.perm(n, 4, B)
    assert not np.array_equal(p, q)
    rec = np.stack([np.arange(n, dtype=np.uint32) ^ 0x55, np.arange(n, dtype=np.uint32)], 1)
    got, _ = oracle.shuffle(rec, 4, B, oracle.BALANCED)
    assert np.array_equal(got, rec[p])
