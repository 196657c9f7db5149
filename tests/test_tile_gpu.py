"""The tile kernel (Fisher-Yates of the base blocks and the first d merge levels on 16-bit
tile-local indices, one CTA of eight warps per tile of 2^d blocks) against the oracle: every
depth it takes, cutoffs that give base blocks of two sizes and uneven merge halves, all element
widths, the per-level tail draws made in the loop when they overflow, the tuned block sizes, the
shuffle's parity pair, and the same calls on the CTA-wide base-block kernel
(MS_FLAG_CTA_TILES)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_1508_03167_gb300 as ms
from paper_1508_03167_gb300 import inputs

pytestmark = pytest.mark.gpu


def _perm(n, seed, B, d, flags=0):
    import torch

    p = ms.params(B, d, flags)
    out = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    nbytes = ms.ms_workspace_bytes(n, 4, p)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = ms.ms_perm(out.data_ptr(), n, seed, ws.data_ptr(), nbytes, p,
                    torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_OK, ms.ms_status_string(st)
    torch.cuda.synchronize()
    return out[:n].cpu().numpy().view(np.uint32)


def _shuffle(arr, seed, B, d, flags=0):
    import torch

    n = arr.shape[0]
    w = arr.nbytes // n
    p = ms.params(B, d, flags)
    x = torch.from_numpy(arr.view(np.uint8).reshape(n, w).copy()).cuda()
    nbytes = ms.ms_workspace_bytes(n, w, p)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = ms.ms_shuffle(x.data_ptr(), n, w, seed, ws.data_ptr(), nbytes, p,
                       torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_OK, ms.ms_status_string(st)
    torch.cuda.synchronize()
    return x.cpu().numpy().view(arr.dtype).reshape(arr.shape)


@pytest.mark.parametrize("n,B", [(1 << 16, 256), (1 << 20, 256), (262147, 256), (100003, 128),
                                 (65537, 1), (8191, 3), (1000003, 1000), (4133, 64),
                                 (300017, 286)])
def test_tile_perm_every_depth(n, B):
    perm = ms.MS_FLAG_PERM
    for seed in (0, 7, 2**63 + 5):
        want, _ = oracle.perm(n, seed, B)
        for d in range(1, 7):
            plan = ms.plan(n, 4, B=B, fuse_depth=d, flags=perm)
            if plan["fuse_depth"] != d:
                continue  # the depth does not fit (c < d, or the tile is too large)
            got = _perm(n, seed, B, d)
            assert np.array_equal(got, want), (n, B, seed, d)


@pytest.mark.parametrize("w", [4, 8, 16])
@pytest.mark.parametrize("n,B", [(262147, 256), (100003, 64), (300017, 286), (5000, 7)])
def test_tile_shuffle_widths(w, n, B):
    if w == 16:
        arr = inputs.records16(n)
    elif w == 8:
        arr = inputs.values_u64(n, 3)
    else:
        arr = inputs.identity_u32(n) * np.uint32(2654435761)
    want, _ = oracle.shuffle(arr, 5, B)
    for d in (1, 4, 5, 6):
        got = _shuffle(arr, 5, B, d)
        assert np.array_equal(got, want), (w, n, B, d)


def test_tile_kernel_and_cta_kernel_agree():
    n, B = 400009, 128
    want, _ = oracle.perm(n, 3, B)
    for d in (2, 3, 5):
        assert np.array_equal(_perm(n, 3, B, d), want), d
        assert np.array_equal(_perm(n, 3, B, d, ms.MS_FLAG_CTA_TILES), want), d


def test_tile_sequential_tails_and_tiny_blocks():
    """B = 1 gives blocks of one or two elements and merges whose tails often cover the whole
    merge; the tail-draw capacity of a level is then exceeded and the draws are made in the
    loop (the result is identical)."""
    for n in (2, 3, 64, 65, 127, 4099):
        want, _ = oracle.perm(n, 9, 1)
        for d in range(1, 7):
            if ms.plan(n, 4, B=1, fuse_depth=d, flags=ms.MS_FLAG_PERM)["fuse_depth"] != d:
                continue
            assert np.array_equal(_perm(n, 9, 1, d), want), (n, d)


def test_tile_large_blocks_of_the_tuned_scale_rows():
    """The tuned rows of the largest arrays use base blocks of up to 512 (perm) and 573 (16-byte
    records) elements, tiles of 32 blocks: the same shapes on arrays the oracle finishes in
    seconds (Fisher-Yates draws of up to 10-bit slices, tiles above 16,000 elements)."""
    n = (1 << 22) + 7  # c = 13: blocks of 512 and 513
    want, _ = oracle.perm(n, 11, 512)
    assert ms.plan(n, 4, B=512, fuse_depth=5, flags=ms.MS_FLAG_PERM)["fuse_depth"] == 5
    assert np.array_equal(_perm(n, 11, 512, 5), want)
    n = 572 * 4096 + 17  # c = 12: blocks of 572 and 573
    arr = inputs.records16(n)
    want, _ = oracle.shuffle(arr, 11, 572)
    assert ms.plan(n, 16, B=572, fuse_depth=5)["fuse_depth"] == 5
    assert np.array_equal(_shuffle(arr, 11, 572, 5), want)


@pytest.mark.parametrize("lg,w", [(26, 4), (26, 8)])
def test_tile_shuffle_pass_parity_by_fused_pair(lg, w):
    """A shuffle of at least 2^28 bytes whose tile pass would be followed by an even number of
    global passes fuses its last two global levels into one pass (instead of fusing one level
    less in the tile). The result is still that of the definition: the shuffle of the identity
    equals the perm of the same (n, seed, B), whose plan has no fused pair."""
    import torch

    n, B, d, seed = 1 << lg, 512, 5, 13
    sh = ms.plan(n, w, B=B, fuse_depth=d)
    assert sh["fuse_depth"] == d and sh["fused_pairs"] == 1
    assert ms.plan(n, 4, B=B, fuse_depth=d, flags=ms.MS_FLAG_PERM)["fused_pairs"] == 0
    p = ms.params(B, d, 0)
    ref = torch.empty(n, dtype=torch.int32, device="cuda")
    nbytes = max(ms.ms_workspace_bytes(n, w, p), ms.ms_workspace_bytes(n, 4, p))
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = ms.ms_perm(ref.data_ptr(), n, seed, ws.data_ptr(), ws.numel(), p,
                    torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_OK, ms.ms_status_string(st)
    x = torch.arange(n, dtype=torch.int64 if w == 8 else torch.int32, device="cuda")
    if w == 8:
        x = x | (x << 32)  # both halves of a row carry its index
    st = ms.ms_shuffle(x.data_ptr(), n, w, seed, ws.data_ptr(), ws.numel(), p,
                       torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_OK, ms.ms_status_string(st)
    torch.cuda.synchronize()
    if w == 8:
        assert torch.equal((x >> 32).to(torch.int32), ref)
        assert torch.equal((x & 0xFFFFFFFF).to(torch.int32), ref)
    else:
        assert torch.equal(x, ref)
