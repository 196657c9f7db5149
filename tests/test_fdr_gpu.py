"""Fast Dice Roller draws on the GPU (MS_FLAG_FDR): the permutation with every uniform draw made
by Lumbroso's FDR on its own stream, and the random-bit counts of that mode, both against the
oracle's FDR mode on the same (n, seed, B), bit for bit and as integers. Then Table 1's measure
at the paper's sizes: the GPU counts the bits of the FDR-mode run for n = 10^5 .. 10^8 (its
Fisher-Yates row is pinned on the CPU), and FDR spends fewer bits than rejection draws."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import paper_1508_03167_gb300 as ms

pytestmark = pytest.mark.gpu


def _gpu_perm(n, seed, B, flags):
    import torch

    out = torch.empty(n, dtype=torch.int32, device="cuda")
    p = ms.params(B=B, flags=flags)
    ws = torch.empty(ms.ms_workspace_bytes(n, 4, p), dtype=torch.uint8, device="cuda")
    st = ms.ms_perm(out.data_ptr(), n, seed, ws.data_ptr(), ws.numel(), p,
                    torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_OK, ms.ms_status_string(st)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("n,B", [(2, 1), (1000, 3), (65_537, 64), (300_017, 512),
                                 (1 << 20, 1024), (2_000_003, 4096)])
def test_fdr_perm_matches_oracle(n, B):
    for seed in (5, 2**40 + 3):
        want, _ = oracle.perm(n, seed, B, oracle.FDR)
        got = _gpu_perm(n, seed, B, ms.MS_FLAG_FDR)
        assert np.array_equal(got, want), (n, B, seed)


def test_fdr_literal_shuffle_of_records_matches_oracle():
    import torch

    n, B = 123_457, 100
    rng = np.random.default_rng(1)
    arr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint32)
    want, _ = oracle.shuffle(arr, 17, B, oracle.FDR | oracle.LITERAL)
    t = torch.from_numpy(arr.view(np.int32)).to("cuda")
    p = ms.params(B=B, flags=ms.MS_FLAG_FDR | ms.MS_FLAG_LITERAL)
    ws = torch.empty(ms.ms_workspace_bytes(n, 16, p), dtype=torch.uint8, device="cuda")
    assert ms.ms_shuffle(t.data_ptr(), n, 16, 17, ws.data_ptr(), ws.numel(), p,
                         torch.cuda.current_stream().cuda_stream) == ms.MS_OK
    torch.cuda.synchronize()
    assert np.array_equal(t.cpu().numpy().view(np.uint32), want)


@pytest.mark.parametrize("n,B", [(7, 2), (100_003, 1024), (1 << 20, 512), (300_017, 5)])
def test_fdr_random_bits_equal_the_oracle(n, B):
    for seed in (0, 9):
        got = ms.random_bits(n, seed, B=B, flags=ms.MS_FLAG_FDR)
        _, st = oracle.perm(n, seed, B, oracle.FDR)
        want = st.as_dict()
        for k in ms.RANDOM_BIT_FIELDS:
            assert got[k] == want[k], (n, B, seed, k, got[k], want[k])


def test_table1_sizes_fdr_spends_fewer_bits_than_rejection():
    for n in (10**5, 10**6, 10**7, 10**8):
        rej = ms.random_bits(n, 1, B=1024)
        fdr = ms.random_bits(n, 1, B=1024, flags=ms.MS_FLAG_FDR)
        assert fdr["coin_bits"] == rej["coin_bits"]
        assert fdr["total_bits"] < rej["total_bits"]
        # n log2 n + Theta(n) either way
        assert 0.0 < fdr["total_bits"] / n - math.log2(n) < 3.0
