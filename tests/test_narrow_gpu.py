"""1- and 2-byte elements: the single call builds the permutation of the same (n, seed, B) on
the 4-byte path, gathers the elements through it and copies them back. Bit-exact with the
oracle's shuffle of the same bytes (the oracle treats elements as opaque w-byte records)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_1508_03167_gb300 as ms

pytestmark = pytest.mark.gpu


def _gpu_shuffle(arr: np.ndarray, seed: int, B: int, fuse_depth: int = -1, flags: int = 0):
    import torch

    n = arr.shape[0]
    w = arr.dtype.itemsize
    p = ms.params(B, fuse_depth, flags)
    x = torch.from_numpy(arr.view(np.uint8).copy()).cuda()
    nbytes = ms.ms_workspace_bytes(n, w, p)
    assert nbytes > 0
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = ms.ms_shuffle(x.data_ptr(), n, w, seed, ws.data_ptr(), nbytes, p,
                       torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_OK, ms.ms_status_string(st)
    torch.cuda.synchronize()
    return x.cpu().numpy().view(arr.dtype)


def _values(n: int, dtype, salt: int) -> np.ndarray:
    rng = np.random.default_rng(1000 + salt)
    return rng.integers(0, np.iinfo(dtype).max, size=n, dtype=dtype, endpoint=True)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
@pytest.mark.parametrize("n,B", [(2, 1), (5, 3), (1023, 16), (65537, 64), (1000003, 128)])
def test_narrow_shuffle_matches_oracle(dtype, n, B):
    arr = _values(n, dtype, n % 97)
    want, _ = oracle.shuffle(arr, 7, B)
    assert np.array_equal(_gpu_shuffle(arr, 7, B), want)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_narrow_shuffle_is_the_perm_gather(dtype):
    """The result is the input gathered through ms_perm's permutation of the same (n, seed, B),
    at the autotuned B and with the tile kernel and fused levels of that plan."""
    import torch

    n = (1 << 22) + 3
    arr = _values(n, dtype, 5)
    p = ms.resolve(n, dtype().itemsize, B=0)
    got = _gpu_shuffle(arr, 11, p.B, p.fuse_depth, p.flags)
    perm = ms.perm(n, 11, B=p.B, fuse_depth=p.fuse_depth, flags=p.flags)
    torch.cuda.synchronize()
    idx = perm.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, arr[idx])


def test_narrow_host_form_and_trivial_sizes():
    import torch

    n, B = 100003, 32
    arr = _values(n, np.uint16, 9)
    want, _ = oracle.shuffle(arr, 3, B)
    p = ms.params(B)
    h = torch.from_numpy(arr.view(np.int16).copy()).pin_memory()
    nbytes = ms.ms_host_workspace_bytes(n, 2, p)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = ms.ms_shuffle_host(h.data_ptr(), n, 2, 3, ws.data_ptr(), nbytes, p,
                            torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_OK, ms.ms_status_string(st)
    assert np.array_equal(h.numpy().view(np.uint16), want)
    for n0 in (0, 1):
        one = np.array([200], dtype=np.uint8)[:n0]
        assert np.array_equal(_gpu_shuffle(one, 1, 4) if n0 else one, one)


def test_narrow_widths_are_unsupported_in_a_batch():
    p = ms.params(B=64)
    assert ms.ms_batch_workspace_bytes([1000, 2000], 1, p) == 0
