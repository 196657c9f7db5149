"""ms_perm_static: the entry point for callers that cannot allocate device memory.

Such callers own their input and output buffers but cannot obtain more device memory (for example
a plugin whose host application owns every allocation). The entry point keeps its scratch in a
fixed array inside the library. Here it is called through the C ABI twice in a row, with different
sizes and seeds, and each result must equal ms_perm's (bit for bit, the tolerance every parity
test of this suite uses). The file is named to be collected last, and passes both alone in a
fresh process and after the rest of the suite.
"""
from __future__ import annotations

import numpy as np
import pytest

import paper_1508_03167_gb300 as ms

pytestmark = pytest.mark.gpu


def _perm_with_workspace(torch, n, seed, p):
    out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    nbytes = ms.ms_workspace_bytes(n, 4, p)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = ms.ms_perm(out.data_ptr(), n, seed, ws.data_ptr(), nbytes, p,
                    torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_OK, ms.ms_status_string(st)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _perm_static(torch, n, seed, p):
    out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    st = ms.ms_perm_static(out.data_ptr(), n, seed, p, torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_OK, ms.ms_status_string(st)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_static_scratch_matches_workspace_path_twice_in_a_row():
    import torch

    calls = [(1 << 20, 1, ms.params(B=1024)),      # the small plain workload
             (300_017, 5, ms.params(B=64))]        # different plan on the same scratch
    for n, seed, p in calls:
        want = _perm_with_workspace(torch, n, seed, p)
        got = _perm_static(torch, n, seed, p)
        assert np.array_equal(got, want), (n, seed)
        assert np.array_equal(np.sort(got.view(np.uint32)), np.arange(n, dtype=np.uint32))


def test_static_entry_point_rejects_sizes_beyond_its_scratch():
    import torch

    out = torch.empty(8, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert ms.ms_perm_static(out.data_ptr(), ms.MS_STATIC_MAX_N + 1, 1, None, s) == \
        ms.MS_ERR_UNSUPPORTED
    # within the size limit but a plan whose scratch does not fit the fixed array
    big = ms.params(B=1, fuse_depth=0, flags=ms.MS_FLAG_GLOBAL_LEVELS)
    assert ms.ms_workspace_bytes(1 << 20, 4, big) > ms.MS_STATIC_SCRATCH_BYTES
    assert ms.ms_perm_static(out.data_ptr(), 1 << 20, 1, big, s) == ms.MS_ERR_UNSUPPORTED


def test_static_entry_point_at_its_size_limit():
    """n = MS_STATIC_MAX_N with the default cutoff: the plan's scratch (one data pass per global
    level, the default for 4-byte elements) fits the fixed array, and the result matches
    ms_perm."""
    import torch

    n = ms.MS_STATIC_MAX_N
    p = ms.params(B=1024)
    assert ms.ms_workspace_bytes(n, 4, p) <= ms.MS_STATIC_SCRATCH_BYTES
    want = _perm_with_workspace(torch, n, 3, p)
    got = _perm_static(torch, n, 3, p)
    assert np.array_equal(got, want)


def test_static_entry_point_runs_fused_pairs_from_its_scratch():
    """At n = MS_STATIC_MAX_N the plan with fused pairs of levels (their exception bitmap, the
    exception lists in patch and in position order, and the rank index) fits the fixed array, so
    the pairs run from it and give the same permutation as ms_perm with its own workspace."""
    import torch

    n = ms.MS_STATIC_MAX_N
    p = ms.params(B=1024, flags=ms.MS_FLAG_PAIR_LEVELS)
    assert ms.ms_workspace_bytes(n, 4, p) <= ms.MS_STATIC_SCRATCH_BYTES
    assert ms.plan(n, 4, B=1024, flags=ms.MS_FLAG_PAIR_LEVELS)["fused_pairs"] > 0
    want = _perm_with_workspace(torch, n, 11, p)
    got = _perm_static(torch, n, 11, p)
    assert np.array_equal(got, want)
