"""Host-side checks of the autotuner: the B = 0 lookup of the C library (built-in table,
installed tables, size buckets, batch median), the table's header round trip and the tuner's
choice rule. No GPU compute."""
from __future__ import annotations

import pytest

import paper_1508_03167_gb300 as ms
from paper_1508_03167_gb300 import tune


@pytest.fixture(autouse=True)
def _restore_builtin_table():
    yield
    ms.ms_tune_install([])


def test_builtin_table_matches_its_header():
    with open(tune.HEADER) as f:
        rows = tune.parse_header(f.read())
    assert rows == ms.ms_tune_table()
    widths = {(r["w"], r["batch"]) for r in rows}
    assert widths == {(w, b) for w in (4, 8, 16) for b in (0, 1)}


def test_explicit_B_is_kept():
    r = ms.resolve(1 << 20, 4, B=333, fuse_depth=2, flags=ms.MS_FLAG_CTA_LEVELS)
    assert (r.B, r.fuse_depth, r.flags) == (333, 2, ms.MS_FLAG_CTA_LEVELS)


def test_buckets_pick_the_smallest_covering_row():
    ms.ms_tune_install([
        dict(w=4, batch=0, log2n_max=24, B=256, fuse_depth=0, flags=0),
        dict(w=4, batch=0, log2n_max=16, B=512, fuse_depth=-1, flags=ms.MS_FLAG_CTA_LEVELS),
        dict(w=4, batch=1, log2n_max=64, B=64, fuse_depth=-1, flags=0),
    ])
    assert ms.resolve(1 << 16, 4, B=0).B == 512          # ceil(log2 n) = 16
    assert ms.resolve((1 << 16) + 1, 4, B=0).B == 256    # 17
    assert ms.resolve(1 << 24, 4, B=0).B == 256
    assert ms.resolve(1 << 30, 4, B=0).B == 256          # beyond every bucket: the largest
    r = ms.resolve(1000, 4, B=0)
    assert r.flags == ms.MS_FLAG_CTA_LEVELS and r.fuse_depth == -1
    # a caller's own level-mode flag and fusion depth win over the table's (B: the row's 512
    # as a block size, 1000 / 2 = 500 being nearer to it than 1000)
    r = ms.resolve(1000, 4, B=0, fuse_depth=1, flags=ms.MS_FLAG_GLOBAL_LEVELS)
    assert (r.B, r.fuse_depth, r.flags) == (500, 1, ms.MS_FLAG_GLOBAL_LEVELS)
    # no row for w = 8: B = 1024
    assert ms.resolve(1 << 20, 8, B=0).B == 1024
    assert ms.resolve_batch([10, 1 << 20, 5], 4, B=0).B == 64


def test_row_B_is_a_block_size():
    """A single call resolves the row's B to the block size floor(n / 2^c) nearest to it by
    ratio; that B gives the listing's cutoff the same c, and n of a power of two times B keeps
    B itself."""
    ms.ms_tune_install([dict(w=16, batch=0, log2n_max=64, B=512, fuse_depth=5, flags=0),
                        dict(w=16, batch=1, log2n_max=64, B=512, fuse_depth=-1, flags=0)])

    def cutoff_levels(n, B):
        c = 0
        while (n >> c) > B:
            c += 1
        return c

    for n, want in [(300_000_017, 572), (1 << 28, 512), (5 << 24, 640), (402_653_184, 384),
                    (700_000, 683), (512, 512), (100, 512), (1025, 512)]:
        r = ms.resolve(n, 16, B=0)
        assert r.B == want, (n, r.B)
        c = cutoff_levels(n, r.B)
        if n > 512:
            assert n >> c == r.B  # blocks of B and B + 1 elements
            # nearest by ratio among the two neighbouring cutoffs
            lo, hi = n >> (c + 1), n >> max(c - 1, 0)
            assert max(r.B, 512) / min(r.B, 512) <= max(lo, 512) / min(lo, 512) or lo == 0
            assert max(r.B, 512) / min(r.B, 512) <= max(hi, 512) / min(hi, 512) or c == 0
        assert ms.plan(n, 16, B=0)["B"] == r.B
    # a batch keeps the row's value
    assert ms.resolve_batch([300_000_017] * 3, 16, B=0).B == 512


def test_tuner_times_a_candidate_at_the_cutoff_its_row_gives():
    # the 300,000,017-record size point: a row of 512 runs with blocks of 572, not the 286 that
    # the cutoff 512 itself gives; at the other points (2^k, 2^k + 17) the two agree
    assert tune.row_cutoff(300_000_017, 16, 512) == 572
    assert tune.row_cutoff((1 << 26) + 17, 16, 512) == 512
    assert tune.row_cutoff(1 << 30, 4, 256) == 256
    # and the built-in table is back in place afterwards
    assert ms.ms_tune_table() == tune.parse_header(open(tune.HEADER).read())


def test_batch_resolves_by_the_median():
    ms.ms_tune_install([
        dict(w=4, batch=1, log2n_max=10, B=32, fuse_depth=-1, flags=0),
        dict(w=4, batch=1, log2n_max=64, B=256, fuse_depth=-1, flags=0),
    ])
    assert ms.resolve_batch([100, 200, 1 << 25], 4, B=0).B == 32
    assert ms.resolve_batch([100, 1 << 20, 1 << 25], 4, B=0).B == 256


def test_plan_and_workspace_use_the_resolved_B():
    r = ms.resolve(1 << 22, 4, B=0)
    assert ms.plan(1 << 22, 4, B=0)["B"] == r.B
    assert ms.ms_workspace_bytes(1 << 22, 4, ms.params(B=0)) == \
        ms.ms_workspace_bytes(1 << 22, 4, r)


def test_malformed_rows_are_rejected():
    for bad in (dict(w=3, batch=0, log2n_max=10, B=64, fuse_depth=-1, flags=0),
                dict(w=4, batch=2, log2n_max=10, B=64, fuse_depth=-1, flags=0),
                dict(w=4, batch=0, log2n_max=10, B=0, fuse_depth=-1, flags=0),
                dict(w=4, batch=0, log2n_max=10, B=ms.MS_MAX_B + 1, fuse_depth=-1, flags=0),
                dict(w=4, batch=0, log2n_max=10, B=64, fuse_depth=-1, flags=ms.MS_FLAG_PERM)):
        with pytest.raises(ms.MsError):
            ms.ms_tune_install([bad])
    assert ms.ms_tune_table() == tune.parse_header(open(tune.HEADER).read())


def test_header_round_trip_and_choice_rule():
    rows = [dict(w=4, batch=0, log2n_max=12, B=64, fuse_depth=-1, flags=8),
            dict(w=16, batch=1, log2n_max=64, B=1024, fuse_depth=0, flags=0)]
    assert tune.parse_header(tune.header_text(rows)) == rows
    assert tune.pick({("a",): [3.0, 1.0, 2.0], ("b",): [1.5, 1.5, 9.0]}) == ("b",)
    assert tune.pick({("a",): [1.0], ("b",): [1.0]}) == ("a",)
    assert tune.buckets([10, 14, 18]) == [12, 16, 64]
