"""Random-bit accounting on the GPU (ms_random_bits) against the oracle's count for the same
(n, seed, B): coin bits (T + 1 per merge), the bits of Algorithm 1's draws and of the merge
tails' draws, draws, merges and leftover, equal as integers. At 2^30 the total follows the
random-bit model: n log2 n + Theta(n) bits."""
from __future__ import annotations

import math

import pytest

import oracle
import paper_1508_03167_gb300 as ms

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,B", [(2, 1), (7, 2), (1000, 3), (65536, 256), (262147, 256),
                                 (100003, 1024), (1 << 20, 1024), (300017, 5)])
def test_random_bits_equal_the_oracle(n, B):
    for seed in (0, 7, 2**63 + 5):
        got = ms.random_bits(n, seed, B=B)
        _, st = oracle.perm(n, seed, B)
        want = st.as_dict()
        for k in ms.RANDOM_BIT_FIELDS:
            assert got[k] == want[k], (n, B, seed, k, got[k], want[k])


def test_random_bits_at_scale_follow_the_model():
    n = 1 << 30
    r = ms.resolve(n, 4, B=0)
    got = ms.random_bits(n, 7, B=r.B)
    per = got["total_bits"] / n
    # n log2 n + Theta(n): the excess per element stays a small constant
    assert 1.0 < per - math.log2(n) < 5.0, per
    assert got["levels"] == ms.plan(n, 4, B=r.B)["c"]
