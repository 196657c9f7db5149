"""GPU <-> oracle parity through the C ABI: bit-exact on every seed, size, cutoff and width.

Sizes span several tiles and ragged tails (non-power-of-two n gives base blocks of two sizes and
uneven merge halves at every level). The result must not depend on the fusion depth, the tile
size or the tail strategy: only (input, n, seed, B) define it."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_1508_03167_gb300 as ms
from paper_1508_03167_gb300 import inputs

pytestmark = pytest.mark.gpu


def _torch():
    import torch

    return torch


def gpu_perm(n: int, seed: int, B: int, fuse_depth: int = -1, flags: int = 0,
             tile_bytes: int = 0) -> np.ndarray:
    torch = _torch()
    p = ms.params(B, fuse_depth, flags, tile_bytes)
    out = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    nbytes = ms.ms_workspace_bytes(n, 4, p)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = ms.ms_perm(out.data_ptr(), n, seed, ws.data_ptr(), nbytes, p,
                    torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_OK, ms.ms_status_string(st)
    torch.cuda.synchronize()
    return out[:n].cpu().numpy().view(np.uint32)


def gpu_shuffle(arr: np.ndarray, seed: int, B: int, fuse_depth: int = -1, flags: int = 0,
                tile_bytes: int = 0) -> np.ndarray:
    torch = _torch()
    n = arr.shape[0]
    w = arr.nbytes // n
    p = ms.params(B, fuse_depth, flags, tile_bytes)
    x = torch.from_numpy(arr.view(np.uint8).reshape(n, w).copy()).cuda()
    nbytes = ms.ms_workspace_bytes(n, w, p)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = ms.ms_shuffle(x.data_ptr(), n, w, seed, ws.data_ptr(), nbytes, p,
                       torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_OK, ms.ms_status_string(st)
    torch.cuda.synchronize()
    return x.cpu().numpy().view(arr.dtype).reshape(arr.shape)


SIZES = [2, 3, 7, 31, 32, 33, 100, 1000, 1023, 1024, 1025, 2047, 2049, 4097, 10007, 65537,
         100003, 262147]


@pytest.mark.parametrize("B", [1, 3, 16, 64, 1024])
def test_perm_matches_oracle_sweep(B):
    for n in SIZES:
        for seed in (0, 7, 2**63 + 5):
            want, _ = oracle.perm(n, seed, B)
            got = gpu_perm(n, seed, B)
            assert np.array_equal(got, want), (n, B, seed)


def test_perm_c1_workload():
    """perm(2^20) of the identity, seed 1, B = 1024 (the small configuration)."""
    want, _ = oracle.perm(1 << 20, 1, 1024)
    got = gpu_perm(1 << 20, 1, 1024)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("n,B", [(1 << 20, 1024), (100003, 16), (262147, 5), (4133, 1)])
def test_result_independent_of_fusion_depth_and_tiles(n, B):
    want, _ = oracle.perm(n, 11, B)
    for d in (0, 1, 2, 3, 5):
        assert np.array_equal(gpu_perm(n, 11, B, fuse_depth=d), want), d
    for tb in (4096, 16384, 98304):
        assert np.array_equal(gpu_perm(n, 11, B, tile_bytes=tb), want), tb


@pytest.mark.parametrize("n,B", [(1 << 20, 1024), (262147, 16), (100003, 256), (65537, 1)])
def test_global_and_local_levels_agree(n, B):
    """Small merge levels normally finish inside one CTA; forcing every level through the
    global plan (chunk prefixes, hash-table tails, patches) must give the same output."""
    want, _ = oracle.perm(n, 13, B)
    assert np.array_equal(gpu_perm(n, 13, B, flags=ms.MS_FLAG_GLOBAL_LEVELS), want)
    assert np.array_equal(gpu_perm(n, 13, B, fuse_depth=0, flags=ms.MS_FLAG_GLOBAL_LEVELS), want)
    assert np.array_equal(gpu_perm(n, 13, B, fuse_depth=0), want)
    assert np.array_equal(gpu_perm(n, 13, B, fuse_depth=0, flags=ms.MS_FLAG_CTA_LEVELS), want)
    assert np.array_equal(gpu_perm(n, 13, B, fuse_depth=0, flags=ms.MS_FLAG_WARP_LEVELS), want)
    assert np.array_equal(gpu_perm(n, 13, B, fuse_depth=0, flags=ms.MS_FLAG_SINGLE_STREAM), want)


@pytest.mark.parametrize("B", [2, 31, 32, 33, 100, 256, 1000, 4096])
def test_fisher_yates_only_base_kernel(B):
    """fuse_depth = 0: the base-block kernel only shuffles blocks (one lane per block)."""
    for n in (B * 37 + 5, 262147):
        want, _ = oracle.perm(n, 21, B)
        assert np.array_equal(gpu_perm(n, 21, B, fuse_depth=0), want), n
    rec = inputs.records16(100003)
    want, _ = oracle.shuffle(rec, 4, B)
    assert np.array_equal(gpu_shuffle(rec, 4, B, fuse_depth=0), want)


@pytest.mark.parametrize("n,B", [(1 << 20, 1024), (262147, 16), (65537, 1)])
def test_sequential_tail_path_is_identical(n, B):
    want, _ = oracle.perm(n, 3, B)
    got = gpu_perm(n, 3, B, fuse_depth=0,
                   flags=ms.MS_FLAG_TAIL_SEQUENTIAL | ms.MS_FLAG_GLOBAL_LEVELS)
    assert np.array_equal(got, want)
    # the streamed small-merge levels' own sequential fallback
    got = gpu_perm(n, 3, B, fuse_depth=0, flags=ms.MS_FLAG_TAIL_SEQUENTIAL)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("w", [4, 8, 16])
@pytest.mark.parametrize("n,B", [(5, 2), (1000, 3), (4099, 64), (100003, 1024), (300017, 1024)])
def test_shuffle_widths_match_oracle(w, n, B):
    if w == 16:
        arr = inputs.records16(n)
    elif w == 8:
        arr = inputs.values_u64(n, 3)
    else:
        arr = inputs.identity_u32(n) * np.uint32(2654435761)
    want, _ = oracle.shuffle(arr, 5, B)
    got = gpu_shuffle(arr, 5, B)
    assert np.array_equal(got, want)


def test_shuffle_is_data_oblivious_on_gpu():
    n, B, seed = 300017, 1024, 9
    rec = inputs.records16(n)
    p = gpu_perm(n, seed, B)
    got = gpu_shuffle(rec, seed, B)
    assert np.array_equal(got, rec[p])


def test_edge_sizes():
    for n in (0, 1):
        assert gpu_perm(n, 1, 4).tolist() == list(range(n))
    # n exactly B, B + 1, 2B, 2B + 1
    for n in (64, 65, 128, 129):
        want, _ = oracle.perm(n, 2, 64)
        assert np.array_equal(gpu_perm(n, 2, 64), want)


@pytest.mark.parametrize("n", [1000, 100003, 1 << 20])
def test_autotuned_B_matches_oracle_at_the_resolved_B(n):
    """B = 0 runs with the tuning table's B; the oracle with that B gives the same result."""
    r = ms.resolve(n, 4, B=0)
    assert r.B >= 1
    got = gpu_perm(n, 11, 0)
    want, _ = oracle.perm(n, 11, r.B)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("n,B", [(1 << 20, 1024), (262147, 16), (100003, 3), (65537, 1),
                                 (1000003, 64)])
def test_fused_level_pairs_match_single_levels(n, B):
    """Consecutive global levels share one data pass (the first level's tail moves become
    exceptions of the second level's gather); one pass per level, the unfused device-side
    fallback (forced by the sequential-tail flag) and the oracle all agree."""
    want, _ = oracle.perm(n, 17, B)
    pl = ms.MS_FLAG_PAIR_LEVELS
    assert ms.plan(n, 4, B=B, fuse_depth=0, flags=pl | ms.MS_FLAG_GLOBAL_LEVELS)["fused_pairs"] > 0
    assert np.array_equal(gpu_perm(n, 17, B, fuse_depth=0, flags=pl), want)
    assert np.array_equal(gpu_perm(n, 17, B, fuse_depth=0, flags=ms.MS_FLAG_SINGLE_LEVELS), want)
    assert np.array_equal(gpu_perm(n, 17, B, fuse_depth=0, flags=pl | ms.MS_FLAG_GLOBAL_LEVELS),
                          want)
    assert np.array_equal(
        gpu_perm(n, 17, B, fuse_depth=0,
                 flags=pl | ms.MS_FLAG_GLOBAL_LEVELS | ms.MS_FLAG_TAIL_SEQUENTIAL), want)


@pytest.mark.parametrize("w", [8, 16])
def test_fused_level_pairs_wide_elements(w):
    n, B = 300017, 16
    arr = inputs.records16(n) if w == 16 else inputs.values_u64(n, 3)
    want, _ = oracle.shuffle(arr, 9, B)
    pl = ms.MS_FLAG_PAIR_LEVELS
    assert np.array_equal(
        gpu_shuffle(arr, 9, B, fuse_depth=0, flags=pl | ms.MS_FLAG_GLOBAL_LEVELS), want)
    assert np.array_equal(gpu_shuffle(arr, 9, B, fuse_depth=0, flags=pl), want)
    assert np.array_equal(gpu_shuffle(arr, 9, B, fuse_depth=0, flags=ms.MS_FLAG_SINGLE_LEVELS),
                          want)
    # the device-side unfused fallback of every pair (forced by the sequential-tail flag)
    assert np.array_equal(
        gpu_shuffle(arr, 9, B, fuse_depth=0,
                    flags=pl | ms.MS_FLAG_GLOBAL_LEVELS | ms.MS_FLAG_TAIL_SEQUENTIAL), want)


def test_concurrent_calls_on_two_streams_from_two_threads():
    """Two host threads call the library at once, each on its own stream (each caller stream gets
    its own plan stream and events); both results equal the oracle's."""
    import threading

    torch = _torch()
    jobs = [(1 << 20, 5, 128), (700001, 6, 64)]
    outs = {}

    def work(i, n, seed, B):
        s = torch.cuda.Stream()
        p = ms.params(B=B, fuse_depth=0)
        out = torch.empty(n, dtype=torch.int32, device="cuda")
        ws = torch.empty(ms.ms_workspace_bytes(n, 4, p), dtype=torch.uint8, device="cuda")
        for _ in range(3):
            assert ms.ms_perm(out.data_ptr(), n, seed, ws.data_ptr(), ws.numel(), p,
                              s.cuda_stream) == ms.MS_OK
        s.synchronize()
        outs[i] = out.cpu().numpy().view(np.uint32)

    th = [threading.Thread(target=work, args=(i, *j)) for i, j in enumerate(jobs)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for i, (n, seed, B) in enumerate(jobs):
        want, _ = oracle.perm(n, seed, B)
        assert np.array_equal(outs[i], want), i


def test_single_call_replays_from_a_cuda_graph():
    """ms_perm and ms_shuffle (global levels, their plans on the paired stream, fused pairs for
    records) captured into one CUDA graph after an eager call on the same stream; replays give
    the oracle's results."""
    torch = _torch()
    n, B = (1 << 20) + 3, 128
    rec = inputs.records16(300017)
    p = ms.params(B=B, fuse_depth=0)
    q = ms.params(B=B, fuse_depth=0, flags=ms.MS_FLAG_PAIR_LEVELS)
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    x = torch.from_numpy(rec.view(np.uint8).reshape(rec.shape[0], 16).copy()).cuda()
    x0 = x.clone()
    ws1 = torch.empty(ms.ms_workspace_bytes(n, 4, p), dtype=torch.uint8, device="cuda")
    ws2 = torch.empty(ms.ms_workspace_bytes(rec.shape[0], 16, q), dtype=torch.uint8,
                      device="cuda")
    s = torch.cuda.Stream()

    def work():
        assert ms.ms_perm(out.data_ptr(), n, 21, ws1.data_ptr(), ws1.numel(), p,
                          s.cuda_stream) == ms.MS_OK
        assert ms.ms_shuffle(x.data_ptr(), rec.shape[0], 16, 22, ws2.data_ptr(), ws2.numel(), q,
                             s.cuda_stream) == ms.MS_OK

    with torch.cuda.stream(s):
        work()  # eager: creates the paired plan stream and sets kernel attributes
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    x.copy_(x0)
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        work()
    want_p, _ = oracle.perm(n, 21, B)
    want_r, _ = oracle.shuffle(rec, 22, B)
    for _ in range(2):
        out.fill_(-1)
        x.copy_(x0)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint32), want_p)
        assert np.array_equal(x.cpu().numpy().view(rec.dtype).reshape(rec.shape), want_r)


@pytest.mark.parametrize("fd", [0, 5])
def test_element_aligned_buffers(fd):
    """The API asks only for w-aligned data: buffers 4 (w = 4) or 8 (w = 8) bytes past a 16-byte
    boundary take the element-wise heads and tails of the staged copies and 16-byte stores, in
    every pass that lands in the caller's buffer."""
    torch = _torch()
    stream = torch.cuda.current_stream().cuda_stream
    for n, B in ((262147, 256), (100003, 64)):
        want, _ = oracle.perm(n, 5, B)
        p = ms.params(B, fd, 0)
        raw = torch.zeros(n + 4, dtype=torch.int32, device="cuda")
        ws = torch.empty(ms.ms_workspace_bytes(n, 4, p), dtype=torch.uint8, device="cuda")
        st = ms.ms_perm(raw.data_ptr() + 4, n, 5, ws.data_ptr(), ws.numel(), p, stream)
        assert st == ms.MS_OK, ms.ms_status_string(st)
        torch.cuda.synchronize()
        got = raw[1:n + 1].cpu().numpy().view(np.uint32)
        assert np.array_equal(got, want), (n, B, fd)
        for w, off in ((4, 4), (8, 8), (8, 24)):
            arr = inputs.values_u64(n, 3) if w == 8 else inputs.identity_u32(n) * np.uint32(2654435761)
            want_s, _ = oracle.shuffle(arr, 5, B)
            nb = arr.nbytes
            buf = torch.zeros(nb + 64, dtype=torch.uint8, device="cuda")
            buf[off:off + nb] = torch.from_numpy(arr.view(np.uint8).copy()).cuda()
            ws = torch.empty(ms.ms_workspace_bytes(n, w, p), dtype=torch.uint8, device="cuda")
            st = ms.ms_shuffle(buf.data_ptr() + off, n, w, 5, ws.data_ptr(), ws.numel(), p, stream)
            assert st == ms.MS_OK, ms.ms_status_string(st)
            torch.cuda.synchronize()
            got_s = buf[off:off + nb].cpu().numpy().view(arr.dtype)
            assert np.array_equal(got_s, want_s), (n, B, fd, w, off)
