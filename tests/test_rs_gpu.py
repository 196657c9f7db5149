"""The splitting process (Rao-Sandelius with a Fisher-Yates cutoff B) through the C ABI,
compared element by element with the CPU oracle on the same (n, seed, B): ragged sizes that span
many 4096-position chunks, cutoffs from 1 (segments of one or two elements, thousands of
segments in a chunk) to 4096, element widths 4, 8 and 16, the perm's generated first level,
n <= B (Fisher-Yates alone), and the trivial sizes."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_1508_03167_gb300 as ms

pytestmark = pytest.mark.gpu


def _torch():
    import torch

    return torch


def _gpu_rs_perm(n, seed, B):
    torch = _torch()
    out = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    nbytes = ms.ms_rs_workspace_bytes(n, 4, B)
    assert nbytes > 0
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = ms.ms_rs_perm(out.data_ptr(), n, seed, B, ws.data_ptr(), nbytes,
                       torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_OK, ms.ms_status_string(st)
    torch.cuda.synchronize()
    return out[:n].cpu().numpy().view(np.uint32)


def _gpu_rs_shuffle(arr, seed, B):
    torch = _torch()
    t = torch.from_numpy(np.ascontiguousarray(arr).view(np.int32)).to("cuda")
    n = arr.shape[0]
    w = arr.nbytes // n
    nbytes = ms.ms_rs_workspace_bytes(n, w, B)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = ms.ms_rs_shuffle(t.data_ptr(), n, w, seed, B, ws.data_ptr(), nbytes,
                          torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_OK, ms.ms_status_string(st)
    torch.cuda.synchronize()
    return t.cpu().numpy().view(arr.dtype).reshape(arr.shape)


@pytest.mark.parametrize("n,B", [(2, 1), (3, 1), (17, 1), (1000, 1), (4097, 2), (10_007, 7),
                                 (65_537, 64), (300_017, 512), (1_000_003, 1000),
                                 (262_147, 4096), (4096 * 3, 255)])
def test_rs_perm_matches_oracle(n, B):
    for seed in (1, 12345678901):
        want, _ = oracle.rs_perm(n, seed, B)
        got = _gpu_rs_perm(n, seed, B)
        assert np.array_equal(got, want), (n, B, seed, int(np.flatnonzero(got != want)[0]))


@pytest.mark.parametrize("n,B", [(1, 1), (5, 8), (4096, 4096), (3000, 4096)])
def test_rs_perm_at_or_below_the_cutoff_is_fisher_yates(n, B):
    want, st = oracle.rs_perm(n, 3, B)
    assert st.merges == 0
    assert np.array_equal(_gpu_rs_perm(n, 3, B), want)


@pytest.mark.parametrize("w,n,B", [(8, 100_003, 128), (16, 70_001, 300), (16, 5000, 4096),
                                   (8, 33, 1)])
def test_rs_shuffle_widths_match_oracle(w, n, B):
    rng = np.random.default_rng(w + n)
    arr = rng.integers(0, 2**32, size=(n, w // 4), dtype=np.uint32)
    want, _ = oracle.rs_shuffle(arr, 9, B)
    got = _gpu_rs_shuffle(arr, 9, B)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("w", [4, 8])
def test_rs_shuffle_of_a_buffer_not_16_byte_aligned(w):
    """The split passes copy a chunk's rows into shared memory 16 bytes at a time when the
    source allows it and an element at a time otherwise: the caller's buffer starts w bytes past
    a 16-byte boundary, the workspace is 256-byte aligned, so the levels alternate the two."""
    torch = _torch()
    n, B, seed = 300_007, 64, 21
    rng = np.random.default_rng(w)
    arr = rng.integers(0, 2**32, size=(n, w // 4), dtype=np.uint32)
    want, _ = oracle.rs_shuffle(arr, seed, B)
    big = torch.from_numpy(np.concatenate([np.zeros(w // 4, np.uint32), arr.reshape(-1)])
                           .view(np.int32)).to("cuda")
    assert big.data_ptr() % 16 == 0
    ptr = big.data_ptr() + w
    nbytes = ms.ms_rs_workspace_bytes(n, w, B)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = ms.ms_rs_shuffle(ptr, n, w, seed, B, ws.data_ptr(), nbytes,
                          torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_OK, ms.ms_status_string(st)
    torch.cuda.synchronize()
    got = big.cpu().numpy().view(np.uint32)[w // 4:].reshape(n, w // 4)
    assert np.array_equal(got, want)


def test_rs_shuffle_is_the_input_gathered_by_the_perm():
    n, B, seed = 2_000_003, 512, 77
    perm = _gpu_rs_perm(n, seed, B)
    arr = np.stack([np.arange(n, dtype=np.uint32), np.arange(n, dtype=np.uint32) ^ 0xA5A5A5A5],
                   axis=1)
    got = _gpu_rs_shuffle(arr, seed, B)
    assert np.array_equal(got, arr[perm])


def test_rs_rejects_bad_arguments():
    torch = _torch()
    buf = torch.empty(64, dtype=torch.int32, device="cuda")
    ws = torch.empty(1 << 16, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert ms.ms_rs_workspace_bytes(100, 4, 0) == 0
    assert ms.ms_rs_shuffle(buf.data_ptr(), 64, 12, 1, 4, ws.data_ptr(), ws.numel(), s) == \
        ms.MS_ERR_INVALID
    assert ms.ms_rs_shuffle(buf.data_ptr(), 64, 4, 1, 8192, ws.data_ptr(), ws.numel(), s) == \
        ms.MS_ERR_UNSUPPORTED
    assert ms.ms_rs_perm(buf.data_ptr(), 64, 1, 4, ws.data_ptr(), 16, s) == ms.MS_ERR_INVALID
