"""Serving loop on the GPU: continuous batching under a memory cap. Every request's result is
identical to the single call on that request (bit for bit), admission never exceeds the arena,
and an overload run (offered load above capacity) still terminates with every request served."""
from __future__ import annotations

import pytest

import paper_1508_03167_gb300 as ms
from paper_1508_03167_gb300 import serve

pytestmark = pytest.mark.gpu


def test_results_equal_alone_and_in_the_mix():
    import torch

    reqs = serve.make_requests(rate_hz=50_000, duration_s=0.01, lo_log2=10, hi_log2=18,
                               seed_base=1000)
    assert len(reqs) > 100
    # small arena: admission has to wait for memory to free up
    srv = serve.Server(arena_bytes=224 << 20, B=128, max_inflight=2, max_batch=64,
                       keep_results=True)
    stats = srv.run(reqs, time_limit=120)
    assert stats["completed"] == len(reqs)
    assert stats["arena_peak_bytes"] <= srv.arena_bytes
    for r in reqs:
        alone = ms.perm(r.n, r.seed, B=128)
        assert torch.equal(srv.results[r.rid], alone), r.rid
    lat = stats["latency_s"]
    assert lat["p50"] is not None and 0 <= lat["p50"] <= lat["p99"] <= lat["max"]


def test_overload_run_terminates():
    reqs = serve.make_requests(rate_hz=200_000, duration_s=0.005, lo_log2=12, hi_log2=20,
                               seed_base=7)
    srv = serve.Server(arena_bytes=512 << 20, B=128, max_inflight=2)
    stats = srv.run(reqs, time_limit=300)
    assert stats["completed"] == len(reqs)
    assert stats["arena_peak_bytes"] <= srv.arena_bytes


def test_request_larger_than_the_arena_is_rejected_not_left_pending():
    """A request whose buffers cannot fit even an empty arena is rejected on arrival; the rest
    are served, and the run ends without hitting its time limit."""
    reqs = serve.make_requests(rate_hz=20_000, duration_s=0.002, lo_log2=10, hi_log2=12,
                               seed_base=3)
    huge = serve.Request(rid=len(reqs), n=1 << 24, seed=99, arrival=reqs[-1].arrival)
    srv = serve.Server(arena_bytes=192 << 20, B=128, max_inflight=2)
    assert srv._footprint(huge.n) > srv.arena_bytes
    stats = srv.run(reqs + [huge], time_limit=60)
    assert stats["rejected"] == 1
    assert stats["completed"] == len(reqs)
    assert not stats["time_limit_hit"] and stats["pending_at_end"] == 0
