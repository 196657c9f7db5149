"""Bit-exact parity with the oracle on the workloads the benchmark times, at their full sizes.

The oracle's outputs there take minutes to compute, so ``tests/golden/make_fullsize_digests.py``
(which calls only the oracle and the input generators) stored their SHA-256 digests in
``tests/golden/fullsize_digests.txt``. Each test here runs the GPU path on exactly the same
(n, seed, B) in the launch configuration the benchmark uses (B = 0 resolved by the built-in
tuning table, automatic fusion depth and level modes: the tile kernel, staged gathers and fused
level pairs), hashes the result and compares digests. Each test first checks that the table
still resolves the workload to the B the digest was computed at, so the digests stay tied to
what the benchmark times. Result definition: Algorithm 2 of the paper with the appendix
listing's block split, on the MS-Philox v1 streams.
"""
from __future__ import annotations

import hashlib
import os

import numpy as np
import pytest

import paper_1508_03167_gb300 as ms
from paper_1508_03167_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "fullsize_digests.txt")


def _digests() -> dict:
    rows = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, n, w, seed, B, digest = line.split()
            rows[name] = dict(n=int(n), w=int(w), seed=int(seed), B=int(B), digest=digest)
    return rows


def _sha_device(t) -> str:
    return hashlib.sha256(t.cpu().numpy().tobytes()).hexdigest()


def _perm(torch, n, seed, p):
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    ws = torch.empty(ms.ms_workspace_bytes(n, 4, p), dtype=torch.uint8, device="cuda")
    st = ms.ms_perm(out.data_ptr(), n, seed, ws.data_ptr(), ws.numel(), p,
                    torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_OK, ms.ms_status_string(st)
    torch.cuda.synchronize()
    del ws
    return out


def test_c1_small_workload_digest():
    import torch

    g = _digests()["c1_perm"]
    out = _perm(torch, g["n"], g["seed"], ms.params(B=g["B"]))
    assert _sha_device(out) == g["digest"]


def test_c2a_perm_2p30_digest_at_the_tuned_plan():
    import torch

    g = _digests()["c2a_perm"]
    p = ms.resolve(g["n"], 4, B=0)
    assert p.B == g["B"], "the tuning table no longer resolves perm(2^30) to the pinned B"
    plan = ms.plan(g["n"], 4, B=p.B, fuse_depth=p.fuse_depth, flags=p.flags | ms.MS_FLAG_PERM)
    assert plan["fuse_depth"] > 0 and plan["tile_smem"] > 0  # the tile kernel's first pass
    out = _perm(torch, g["n"], g["seed"], p)
    assert _sha_device(out) == g["digest"]
    del out
    torch.cuda.empty_cache()


def test_c2b_records_3e8_digest_at_the_tuned_plan():
    import torch

    g = _digests()["c2b_records"]
    p = ms.resolve(g["n"], 16, B=0)
    assert p.B == g["B"], "the tuning table no longer resolves the records to the pinned B"
    assert ms.ms_plan_info(g["n"], 16, p).fused_pairs > 0
    rec = torch.from_numpy(inputs.records16(g["n"]).view(np.int32)).to("cuda")
    ws = torch.empty(ms.ms_workspace_bytes(g["n"], 16, p), dtype=torch.uint8, device="cuda")
    st = ms.ms_shuffle(rec.data_ptr(), g["n"], 16, g["seed"], ws.data_ptr(), ws.numel(), p,
                       torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_OK, ms.ms_status_string(st)
    torch.cuda.synchronize()
    del ws
    assert _sha_device(rec) == g["digest"]
    del rec
    torch.cuda.empty_cache()


def test_c3_batched_workload_digest():
    """The 4096 perm(n_i) of the batched workload in one batched call at the batch's B."""
    import torch

    g = _digests()["c3_batch"]
    sizes = [int(x) for x in inputs.batch_sizes_log_uniform(4096, 6, 20)]
    assert sum(sizes) == g["n"]
    B = ms.resolve_batch(sizes, 4, B=0, flags=ms.MS_FLAG_PERM).B
    assert B == g["B"], "the tuning table no longer resolves the batch to the pinned B"
    outs = [torch.empty(n, dtype=torch.int32, device="cuda") for n in sizes]
    p = ms.params(B=B, flags=ms.MS_FLAG_PERM)
    nbytes = ms.ms_batch_workspace_bytes(sizes, 4, p)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = ms.ms_shuffle_batch([o.data_ptr() for o in outs], sizes, 4, None, g["seed"],
                             ws.data_ptr(), nbytes, p, torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_OK, ms.ms_status_string(st)
    torch.cuda.synchronize()
    flat = torch.cat(outs).cpu().numpy()
    h = hashlib.sha256()
    off = 0
    for n in sizes:
        h.update(flat[off:off + n].tobytes())
        off += n
    assert h.hexdigest() == g["digest"]


def test_c4_batched_large_instances_digest():
    """The whole batched-large workload (64 uint64 arrays, 3.26e9 elements) in one batched call;
    its largest instance and its smallest (taken by the persistent engine) match the oracle."""
    import torch

    g = _digests()
    pinned = {int(k.split("_")[-1]): v for k, v in g.items() if k.startswith("c4_u64_")}
    sizes = [int(x) for x in inputs.batch_sizes_uniform(64, 10**6, 10**8)]
    B = ms.resolve_batch(sizes, 8, B=0).B
    assert all(v["B"] == B for v in pinned.values()), "batch B moved from the pinned B"
    bufs = [inputs.values_u64_torch(n, i).view(torch.int64) for i, n in enumerate(sizes)]
    p = ms.params(B=B)
    nbytes = ms.ms_batch_workspace_bytes(sizes, 8, p)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = ms.ms_shuffle_batch([b.data_ptr() for b in bufs], sizes, 8, None, 1, ws.data_ptr(),
                             nbytes, p, torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_OK, ms.ms_status_string(st)
    torch.cuda.synchronize()
    del ws
    for i, v in pinned.items():
        assert sizes[i] == v["n"] and v["seed"] == 1 + i
        assert _sha_device(bufs[i]) == v["digest"], i
    del bufs
    torch.cuda.empty_cache()


def test_rao_sandelius_perm_2p30_digest():
    """The comparison workload the benchmark times: the splitting process's perm of 2^30
    positions, seed 7, cutoff 512."""
    import torch

    g = _digests()["rs_perm"]
    out = torch.empty(g["n"], dtype=torch.int32, device="cuda")
    nbytes = ms.ms_rs_workspace_bytes(g["n"], 4, g["B"])
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = ms.ms_rs_perm(out.data_ptr(), g["n"], g["seed"], g["B"], ws.data_ptr(), nbytes,
                       torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_OK, ms.ms_status_string(st)
    torch.cuda.synchronize()
    del ws
    assert _sha_device(out) == g["digest"]
    del out
    torch.cuda.empty_cache()


def test_max_size_perm_digest():
    """n = 2^32 - 1, the largest n the boundary takes, at its tuned plan (the tile kernel, then
    18 global levels): every 32-bit position and index of the path near its limit. The result
    is hashed from the device in 1 GiB slices."""
    import torch

    g = _digests()["max_perm"]
    p = ms.resolve(g["n"], 4, B=0)
    assert p.B == g["B"], "the tuning table no longer resolves perm(2^32 - 1) to the pinned B"
    out = _perm(torch, g["n"], g["seed"], p)
    h = hashlib.sha256()
    step = 1 << 28
    for i in range(0, g["n"], step):
        h.update(out[i:i + step].cpu().numpy())
    assert h.hexdigest() == g["digest"]
    del out
    torch.cuda.empty_cache()


def test_rao_sandelius_max_size_digest():
    """The splitting process on n = 2^32 - 1 positions (seed 5, cutoff 512): segment bounds,
    chunk and bitmap indices of every split level and of the Fisher-Yates pass near 2^32. The
    result is hashed from the device in 1 GiB slices."""
    import torch

    g = _digests()["rs_max"]
    out = torch.empty(g["n"], dtype=torch.int32, device="cuda")
    nbytes = ms.ms_rs_workspace_bytes(g["n"], 4, g["B"])
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = ms.ms_rs_perm(out.data_ptr(), g["n"], g["seed"], g["B"], ws.data_ptr(), nbytes,
                       torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_OK, ms.ms_status_string(st)
    torch.cuda.synchronize()
    del ws
    h = hashlib.sha256()
    step = 1 << 28
    for i in range(0, g["n"], step):
        h.update(out[i:i + step].cpu().numpy())
    assert h.hexdigest() == g["digest"]
    del out
    torch.cuda.empty_cache()
