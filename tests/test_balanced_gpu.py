"""Merges driven by a balanced word (MS_FLAG_BALANCED) through the C ABI, compared element by
element with the oracle's BALANCED mode on the same (n, seed, B): the word of every merge is its
halves' labels merged by the merge's own coins and insertions (applied to label bytes on the
GPU, by the parallel insertion patches or the sequential fallback), and the data is interleaved
stably by it."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_1508_03167_gb300 as ms

pytestmark = pytest.mark.gpu


def _run(arr, seed, B, flags=0, perm=False):
    import torch

    n = arr.shape[0]
    w = 4 if perm else arr.nbytes // n
    t = (torch.empty(n, dtype=torch.int32, device="cuda") if perm else
         torch.from_numpy(np.ascontiguousarray(arr).view(np.int32)).to("cuda"))
    p = ms.params(B=B, flags=flags | ms.MS_FLAG_BALANCED)
    ws = torch.empty(ms.ms_workspace_bytes(n, w, p), dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    st = (ms.ms_perm(t.data_ptr(), n, seed, ws.data_ptr(), ws.numel(), p, s) if perm else
          ms.ms_shuffle(t.data_ptr(), n, w, seed, ws.data_ptr(), ws.numel(), p, s))
    assert st == ms.MS_OK, ms.ms_status_string(st)
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint32).reshape(arr.shape)


@pytest.mark.parametrize("n,B", [(2, 1), (17, 2), (1000, 1), (65_537, 16), (300_017, 64),
                                 (1 << 20, 1024), (4_000_037, 512)])
def test_balanced_perm_matches_oracle(n, B):
    for seed in (3, 2**33 + 7):
        want, _ = oracle.perm(n, seed, B, oracle.BALANCED)
        got = _run(np.empty(n, dtype=np.uint32), seed, B, perm=True)
        assert np.array_equal(got, want), (n, B, seed, int(np.flatnonzero(got != want)[0]))


@pytest.mark.parametrize("w", [8, 16])
def test_balanced_shuffle_widths_match_oracle(w):
    n, B = 200_003, 128
    arr = np.random.default_rng(w).integers(0, 2**32, size=(n, w // 4), dtype=np.uint32)
    want, _ = oracle.shuffle(arr, 29, B, oracle.BALANCED)
    assert np.array_equal(_run(arr, 29, B), want)


def test_balanced_with_sequential_insertions_and_fdr_draws():
    n, B = 500_009, 256
    want, _ = oracle.perm(n, 31, B, oracle.BALANCED)
    got = _run(np.empty(n, dtype=np.uint32), 31, B, flags=ms.MS_FLAG_TAIL_SEQUENTIAL, perm=True)
    assert np.array_equal(got, want)
    want, _ = oracle.perm(n, 31, B, oracle.BALANCED | oracle.FDR)
    got = _run(np.empty(n, dtype=np.uint32), 31, B, flags=ms.MS_FLAG_FDR, perm=True)
    assert np.array_equal(got, want)


def test_balanced_and_literal_together_are_rejected():
    p = ms.params(B=64, flags=ms.MS_FLAG_BALANCED | ms.MS_FLAG_LITERAL)
    assert ms.ms_workspace_bytes(1000, 4, p) == 0
