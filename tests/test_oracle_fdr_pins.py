"""Pins of the oracle's per-stream Fast Dice Roller draws (mode FDR: every uniform draw of
MS-Philox v1 made by Lumbroso's Fast Dice Roller, the optimal uniform draw Section 1 cites, on the
draw's own Philox stream), against what the mathematics fixes:
  * every value in [0, R) is drawn, with frequencies a chi-square test accepts;
  * the mean bits per draw equal FDR's exact expectation: v doubles with each bit and, once
    v >= R, the draw continues with probability (v - R) / v and v - R;
  * a block at or below the cutoff (plain Fisher-Yates) spends, on average, Table 1's
    Fisher-Yates row at n = 10^5 (the same expectation as a sequential bit stream);
  * the permutation is uniform: Fisher-Yates and the merges are unchanged, only the draws'
    values and costs move (a perm is a permutation; shuffles are data-oblivious)."""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _fdr_expected_bits(R: int) -> float:
    if R <= 1:
        return 0.0
    v, p, e = 1, 1.0, 0.0
    while p > 1e-18:
        v *= 2
        e += p
        if v >= R:
            p *= (v - R) / v
            v -= R
    return e


@pytest.mark.parametrize("R", [2, 3, 5, 7, 100, 1000, 65537])
def test_fdr_draws_are_uniform_and_cost_the_exact_expectation(R):
    trials = 20000
    vals, bits = np.zeros(trials, dtype=np.int64), np.zeros(trials)
    for i in range(trials):
        vals[i], bits[i] = oracle.draw_fdr(3, oracle.TAG_TAIL, 1, 7, i, R)
    assert vals.min() >= 0 and vals.max() < R
    if R <= 100:
        cnt = np.bincount(vals, minlength=R)
        chi2 = ((cnt - trials / R) ** 2 / (trials / R)).sum()
        assert chi2 < R - 1 + 6 * math.sqrt(2 * (R - 1)), chi2
    want = _fdr_expected_bits(R)
    se = bits.std() / math.sqrt(trials)
    assert abs(bits.mean() - want) < 5 * se + 1e-9, (bits.mean(), want)


def test_fdr_fisher_yates_matches_table1_row():
    n, trials = 100_000, 40
    with open(os.path.join(GOLDEN, "table1_random_bits.txt")) as f:
        paper = {(l.split()[0], int(l.split()[1])): int(l.split()[2])
                 for l in f if l.strip() and not l.startswith("#")}[("fisher_yates", n)]
    got = np.array([oracle.perm(n, s, n, oracle.FDR)[1].leaf_bits for s in range(trials)],
                   dtype=float)
    want = sum(_fdr_expected_bits(R) for R in range(2, n + 1))
    sd = got.std()
    assert abs(got.mean() - want) < 5 * sd / math.sqrt(trials), (got.mean(), want)
    assert abs(got.mean() - paper) < 4.5 * math.sqrt(sd ** 2 / trials + sd ** 2 / 100)


@pytest.mark.parametrize("n,B", [(1000, 16), (65_537, 256)])
def test_fdr_mode_keeps_the_coins_and_gives_permutations(n, B):
    p, st = oracle.perm(n, 8, B, oracle.FDR)
    q, st0 = oracle.perm(n, 8, B)
    assert np.array_equal(np.sort(p), np.arange(n, dtype=np.uint32))
    assert st.coin_bits == st0.coin_bits and st.merges == st0.merges
    rec = np.stack([np.arange(n, dtype=np.uint32) * 7, np.arange(n, dtype=np.uint32)], 1)
    got, _ = oracle.shuffle(rec, 8, B, oracle.FDR)
    assert np.array_equal(got, rec[p])


def test_fdr_and_rejection_draws_differ_in_value_and_cost():
    n = 5000
    p, st = oracle.perm(n, 4, n, oracle.FDR)
    q, st0 = oracle.perm(n, 4, n)
    assert not np.array_equal(p, q)
    assert st.leaf_bits < st0.leaf_bits  # FDR spends fewer bits than ceil(log2 R) rejection
