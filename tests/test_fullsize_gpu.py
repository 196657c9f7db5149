"""Full-size checks at the scale workload's sizes and launch configuration (perm of 2^30 uint32
and a shuffle of 300,000,017 16-byte records, seed 7, autotuned B), where the oracle would take
minutes: properties that hold at any size.
  * the 2^30 output is a permutation of 0..n-1;
  * it does not depend on the kernels (no fused levels and every level through the global
    plan gives the same array as the tuned plan, whose tile kernel fuses the first levels);
  * the record shuffle is data-oblivious: its output equals the input gathered by the perm of the
    same (n, seed, B), so the 16-byte path agrees with the 4-byte path element by element."""
from __future__ import annotations

import pytest

import paper_1508_03167_gb300 as ms

pytestmark = pytest.mark.gpu

SEED = 7


def _perm(n, p):
    import torch

    out = torch.empty(n, dtype=torch.int32, device="cuda")
    ws = torch.empty(ms.ms_workspace_bytes(n, 4, p), dtype=torch.uint8, device="cuda")
    st = ms.ms_perm(out.data_ptr(), n, SEED, ws.data_ptr(), ws.numel(), p,
                    torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_OK, ms.ms_status_string(st)
    del ws
    return out


def test_perm_2p30_is_a_permutation_and_level_mode_independent():
    import torch

    n = 1 << 30
    p = ms.resolve(n, 4, B=0)
    out = _perm(n, p)
    seen = torch.zeros(n, dtype=torch.bool, device="cuda")
    seen[out.long()] = True
    assert bool(seen.all())
    del seen
    # the same permutation with no fused levels and every level through the global plan
    q = ms.params(B=p.B, fuse_depth=0, flags=ms.MS_FLAG_GLOBAL_LEVELS)
    assert ms.plan(n, 4, B=p.B, fuse_depth=0, flags=ms.MS_FLAG_GLOBAL_LEVELS)["global_levels"] > \
        ms.ms_plan_info(n, 4, p).global_levels
    other = _perm(n, q)
    assert torch.equal(out, other)
    del out, other
    torch.cuda.empty_cache()


def test_records_3e8_equal_input_gathered_by_perm():
    import torch

    n = 300_000_017
    p = ms.resolve(n, 16, B=0)
    idx = torch.arange(n, dtype=torch.int32, device="cuda")
    rec = torch.stack([idx, idx ^ 0x5BD1E995, idx * 0x01000193, ~idx], dim=1).contiguous()
    src = rec.clone()
    ws = torch.empty(ms.ms_workspace_bytes(n, 16, p), dtype=torch.uint8, device="cuda")
    st = ms.ms_shuffle(rec.data_ptr(), n, 16, SEED, ws.data_ptr(), ws.numel(), p,
                       torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_OK, ms.ms_status_string(st)
    del ws
    perm = _perm(n, ms.params(B=p.B, fuse_depth=p.fuse_depth, flags=p.flags))
    assert torch.equal(rec, src[perm.long()])
    del rec, src, perm, idx
    torch.cuda.empty_cache()
