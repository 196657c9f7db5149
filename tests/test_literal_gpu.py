"""Algorithm 3 as printed (MS_FLAG_LITERAL): the in-place swapping merge, whose first half leaves
in a rotated order, through the C ABI, compared element by element with the oracle's literal mode
on the same (n, seed, B). The sizes span many 4096-step chunks and merges whose first half runs
through many laps of its rotating queue; cutoffs down to 1 give merges whose halves differ by one
and levels with a million merges."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_1508_03167_gb300 as ms

pytestmark = pytest.mark.gpu


def _gpu(arr, seed, B, flags=0):
    import torch

    n = arr.shape[0]
    w = arr.nbytes // n
    t = torch.from_numpy(np.ascontiguousarray(arr).view(np.int32)).to("cuda")
    p = ms.params(B=B, flags=flags | ms.MS_FLAG_LITERAL)
    ws = torch.empty(ms.ms_workspace_bytes(n, w, p), dtype=torch.uint8, device="cuda")
    st = ms.ms_shuffle(t.data_ptr(), n, w, seed, ws.data_ptr(), ws.numel(), p,
                       torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_OK, ms.ms_status_string(st)
    torch.cuda.synchronize()
    return t.cpu().numpy().view(arr.dtype).reshape(arr.shape)


def _gpu_perm(n, seed, B, flags=0):
    import torch

    out = torch.empty(n, dtype=torch.int32, device="cuda")
    p = ms.params(B=B, flags=flags | ms.MS_FLAG_LITERAL)
    ws = torch.empty(ms.ms_workspace_bytes(n, 4, p), dtype=torch.uint8, device="cuda")
    st = ms.ms_perm(out.data_ptr(), n, seed, ws.data_ptr(), ws.numel(), p,
                    torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_OK, ms.ms_status_string(st)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("n,B", [(2, 1), (3, 1), (17, 2), (1000, 1), (65_537, 16),
                                 (300_017, 64), (1 << 20, 1024), (4_000_037, 512),
                                 (1_000_003, 1)])
def test_literal_perm_matches_oracle(n, B):
    for seed in (1, 987654321987):
        want, _ = oracle.perm(n, seed, B, mode=oracle.LITERAL)
        got = _gpu_perm(n, seed, B)
        assert np.array_equal(got, want), (n, B, seed, int(np.flatnonzero(got != want)[0]))


def test_literal_differs_from_the_stable_interleave():
    n, B = 100_003, 64
    lit = _gpu_perm(n, 5, B)
    stable, _ = oracle.perm(n, 5, B)
    assert not np.array_equal(lit, stable)
    assert np.array_equal(np.sort(lit), np.arange(n, dtype=np.uint32))


@pytest.mark.parametrize("w", [8, 16])
def test_literal_shuffle_widths_match_oracle(w):
    n, B = 200_003, 128
    rng = np.random.default_rng(w)
    arr = rng.integers(0, 2**32, size=(n, w // 4), dtype=np.uint32)
    want, _ = oracle.shuffle(arr, 13, B, mode=oracle.LITERAL)
    assert np.array_equal(_gpu(arr, 13, B), want)


def test_literal_with_sequential_tails_is_identical():
    n, B = 500_009, 256
    want, _ = oracle.perm(n, 21, B, mode=oracle.LITERAL)
    got = _gpu_perm(n, 21, B, flags=ms.MS_FLAG_TAIL_SEQUENTIAL)
    assert np.array_equal(got, want)


def test_literal_batch_is_unsupported():
    import torch

    sizes = [1000, 2000]
    bufs = [torch.empty(k, dtype=torch.int32, device="cuda") for k in sizes]
    p = ms.params(B=64, flags=ms.MS_FLAG_PERM | ms.MS_FLAG_LITERAL)
    assert ms.ms_batch_workspace_bytes(sizes, 4, p) == 0
    st = ms.ms_shuffle_batch([b.data_ptr() for b in bufs], sizes, 4, None, 1, 0, 0, p,
                             torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_ERR_UNSUPPORTED
