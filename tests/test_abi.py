"""Host-side checks of the C ABI (no GPU compute): the library loads, exports every entry point
include/mergeshuffle.h declares, plans the configurations of the workloads correctly and rejects
bad arguments synchronously. Also checks that the oracle and the CUDA path share no code."""
from __future__ import annotations

import os
import re

import pytest

import paper_1508_03167_gb300 as ms

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions() -> list[str]:
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(ms_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    lib = ms.lib()
    names = _declared_functions()
    assert "ms_shuffle" in names and "ms_perm" in names
    for name in names:
        assert hasattr(lib, name), name


def test_version_and_status_strings():
    assert "MS-Philox v1" in ms.ms_version()
    assert ms.ms_status_string(ms.MS_OK) == "MS_OK"
    assert ms.ms_status_string(ms.MS_ERR_INVALID) == "MS_ERR_INVALID"


def test_default_params():
    p = ms.ms_default_params()
    assert p.B == 1024 and p.fuse_depth == -1 and p.flags == 0


@pytest.mark.parametrize("n,B,c", [(2**20, 1024, 10), (2**30, 1024, 20), (300_000_017, 1024, 19),
                                   (2049, 1024, 1), (1024, 1024, 0), (5, 1, 2), (8, 1, 3)])
def test_plan_levels_follow_the_cutoff_rule(n, B, c):
    p = ms.ms_plan_info(n, 4, ms.params(B=B))
    assert p.c == c
    assert p.fuse_depth <= c
    assert p.hbm_levels == c - p.fuse_depth
    assert p.passes == 1 + p.hbm_levels - p.fused_pairs
    assert 2 * p.fused_pairs <= p.global_levels
    q = ms.ms_plan_info(n, 4, ms.params(B=B, flags=ms.MS_FLAG_SINGLE_LEVELS))
    assert q.fused_pairs == 0 and q.passes == 1 + q.hbm_levels
    assert p.tiles == (1 << c) >> p.fuse_depth


def test_plan_fusion_depth_and_workspace():
    p = ms.ms_plan_info(2**30, 4, ms.params(B=1024))
    # 48 KiB tiles of 4-byte elements hold 2^13 elements: 8 base blocks of 1024
    assert p.fuse_depth == 3
    assert p.tile_max == 8192
    ws = ms.ms_workspace_bytes(2**30, 4, ms.params(B=1024))
    assert ws >= 2**30 * 4
    # the ping-pong partner plus the plans of two units of global levels in flight
    assert ws < 2**30 * 4 * 1.8
    assert ms.ms_host_workspace_bytes(2**30, 4, ms.params(B=1024)) >= ws + 2**30 * 4
    # forced depth is honoured (capped by c)
    assert ms.ms_plan_info(2**20, 4, ms.params(B=1024, fuse_depth=0)).fuse_depth == 0
    perm = ms.MS_FLAG_PERM
    assert ms.ms_plan_info(2**20, 4, ms.params(B=1024, fuse_depth=2, flags=perm)).fuse_depth == 2
    # a shuffle's tile pass must not run in place: with 1 span level and 7 global
    # levels after it, it fuses one level less (an odd number of passes follows)
    sh = ms.ms_plan_info(2**20, 4, ms.params(B=1024, fuse_depth=2))
    assert sh.fuse_depth == 1 and (sh.passes - 1) % 2 == 1
    # the workspace covers both forms
    for fl in (0, perm):
        assert ms.ms_workspace_bytes(2**20, 4, ms.params(B=1024, fuse_depth=2)) >= \
            ms.ms_plan_info(2**20, 4, ms.params(B=1024, fuse_depth=2, flags=fl)).workspace_bytes
    assert ms.ms_plan_info(3000, 4, ms.params(B=1024, fuse_depth=9, flags=perm)).fuse_depth == 2
    # (all of a shuffle's levels fused would leave its tile pass in place)
    assert ms.ms_plan_info(3000, 4, ms.params(B=1024, fuse_depth=9)).fuse_depth == 1
    # from 2^28 bytes on, the shuffle fuses its last two global levels into one pass instead
    big = ms.ms_plan_info(1 << 26, 4, ms.params(B=512, fuse_depth=5))
    assert big.fuse_depth == 5 and big.fused_pairs == 1 and (big.passes - 1) % 2 == 1
    assert ms.ms_plan_info(1 << 26, 4, ms.params(B=512, fuse_depth=5, flags=perm)).fused_pairs == 0
    # (one level less where single passes are forced)
    single = ms.ms_plan_info(1 << 26, 4, ms.params(B=512, fuse_depth=5,
                                                   flags=ms.MS_FLAG_SINGLE_LEVELS))
    assert single.fuse_depth == 4 and single.fused_pairs == 0


def test_tuned_tile_shapes_keep_their_occupancy():
    """The tile kernel's shared memory at the tuned shapes: B = 512 at 2^30 (tiles of 16,384)
    fits three CTAs in an SM's 228 KB (with 1 KB reserved and at most 2 KB of static shared
    memory a CTA), B = 256 five (the registers allow four), the records' B = 572 two."""
    perm = ms.MS_FLAG_PERM
    per_sm = 228 * 1024

    def ctas(t):
        return per_sm // (t + 1024 + 2048)

    t512 = ms.ms_plan_info(1 << 30, 4, ms.params(B=512, fuse_depth=5, flags=perm)).tile_smem
    t256 = ms.ms_plan_info(1 << 30, 4, ms.params(B=256, fuse_depth=5, flags=perm)).tile_smem
    t572 = ms.ms_plan_info(300_000_017, 16, ms.params(B=572, fuse_depth=5)).tile_smem
    assert (ctas(t512), ctas(t256), ctas(t572)) == (3, 5, 2), (t512, t256, t572)
    # no tile pass, no tile shared memory
    assert ms.ms_plan_info(1 << 20, 4, ms.params(B=1024, fuse_depth=0)).tile_smem == 0
    assert ms.ms_plan_info(1 << 30, 4, ms.params(B=512, fuse_depth=5,
                                                 flags=perm | ms.MS_FLAG_CTA_TILES)).tile_smem == 0


def test_plan_records():
    p = ms.ms_plan_info(300_000_017, 16, ms.params(B=1024))
    assert p.c == 19 and p.w == 16
    assert p.tile_max * 16 <= 48 * 1024


@pytest.mark.parametrize("n,w,B,status", [(100, 3, 16, ms.MS_ERR_INVALID),
                                          (100, 3, 0, ms.MS_ERR_INVALID),
                                          (2**32, 4, 16, ms.MS_ERR_INVALID),
                                          (100, 4, 5000, ms.MS_ERR_UNSUPPORTED)])
def test_invalid_arguments_are_rejected_synchronously(n, w, B, status):
    with pytest.raises(ms.MsError) as e:
        ms.ms_plan_info(n, w, ms.params(B=B))
    assert e.value.status == status
    assert ms.ms_workspace_bytes(n, w, ms.params(B=B)) == 0
    # the compute entry points validate before touching any device state
    assert ms.ms_shuffle(0x1000, n, w, 1, 0, 0, ms.params(B=B), 0) == status


@pytest.mark.parametrize("w", [1, 2])
def test_narrow_widths_size_and_validate_as_a_4_byte_perm(w):
    """1- and 2-byte elements run the 4-byte perm of the same (n, seed, B), then gather through
    it: their workspace is the indices plus the 4-byte workspace, B = 0 resolves as for 4 bytes,
    and bad arguments get the 4-byte path's status."""
    n = 1000003
    p = ms.params(B=64)
    assert ms.ms_workspace_bytes(n, w, p) == ((4 * n + 255) // 256) * 256 + \
        ms.ms_workspace_bytes(n, 4, p)
    assert ms.resolve(n, w, B=0).B == ms.resolve(n, 4, B=0).B
    assert ms.ms_shuffle(0x1000, n, w, 1, 0, 0, ms.params(B=5000), 0) == ms.MS_ERR_UNSUPPORTED
    assert ms.ms_shuffle(0x1000, 2**32, w, 1, 0, 0, ms.params(B=16), 0) == ms.MS_ERR_INVALID
    need = ms.ms_workspace_bytes(n, w, p)
    assert ms.ms_shuffle(0x1000, n, w, 1, 0x10000, need - 1, p, 0) == ms.MS_ERR_INVALID
    assert ms.ms_shuffle(0, 1, w, 1, 0, 0, None, 0) == ms.MS_OK


def test_small_workspace_is_rejected():
    need = ms.ms_workspace_bytes(10**6, 4, ms.params(B=64))
    assert ms.ms_shuffle(0x1000, 10**6, 4, 1, 0x10000, need - 1, ms.params(B=64), 0) == \
        ms.MS_ERR_INVALID
    assert ms.ms_shuffle(0x1002, 10**6, 4, 1, 0x10000, need, ms.params(B=64), 0) == \
        ms.MS_ERR_INVALID  # misaligned data


def test_trivial_sizes_launch_nothing():
    # n <= 1 needs no device work at all for shuffle
    assert ms.ms_shuffle(0, 0, 4, 1, 0, 0, None, 0) == ms.MS_OK
    assert ms.ms_shuffle(0x1000, 1, 16, 1, 0, 0, None, 0) == ms.MS_OK


def test_oracle_and_cuda_path_share_no_code():
    pkg = os.path.join(ROOT, "paper_1508_03167_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "ms_oracle" not in text, f
                assert not re.search(r"^\s*(from|import)\s+oracle\b", text, re.M), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            text = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_1508_03167_gb300" not in text, f
            assert "mergeshuffle.h" not in text, f


def test_plan_invariants_on_random_requests():
    """Planner invariants over seeded random (n, w, B, fuse depth, mode flag) requests: the
    cutoff of the appendix listing (c = min{c : floor(n / 2^c) <= B}), passes = 1 + HBM levels
    - fused pairs, the fusion depth within c, the tile kernel's shared memory within its
    budget, and a shuffle's tile pass never in place (an odd number of passes follows it, so
    the last lands in the caller's array)."""
    import random

    rng = random.Random(5)
    modes = [0, ms.MS_FLAG_PERM, ms.MS_FLAG_SINGLE_LEVELS, ms.MS_FLAG_PAIR_LEVELS,
             ms.MS_FLAG_GLOBAL_LEVELS, ms.MS_FLAG_CTA_TILES]
    tiled = 0
    for _ in range(1500):
        n = min(int(2 ** rng.uniform(1, 32)), 2**32 - 1)
        fl = rng.choice(modes)
        w = 4 if fl == ms.MS_FLAG_PERM else rng.choice([4, 8, 16])
        B = rng.randint(1, ms.MS_MAX_B)
        d = rng.choice([-1, 0, 1, 2, 3, 4, 5, 6])
        p = ms.ms_plan_info(n, w, ms.params(B=B, fuse_depth=d, flags=fl))
        c = 0
        while (n >> c) > B:
            c += 1
        case = (n, w, B, d, fl)
        assert p.c == c, case
        if n <= 1:
            continue
        assert p.passes == 1 + p.hbm_levels - p.fused_pairs, case
        assert p.fuse_depth <= c and p.hbm_levels == c - p.fuse_depth, case
        if p.tile_smem:
            tiled += 1
            assert p.tile_smem <= 200 * 1024, case
            if not fl & ms.MS_FLAG_PERM:
                assert (p.passes - 1) % 2 == 1, case
    assert tiled > 300  # the tile kernel's plans are well represented
