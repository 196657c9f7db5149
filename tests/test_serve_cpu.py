"""Host-side serving logic (no GPU): the device-memory arena used for admission."""
from __future__ import annotations

import random

from paper_1508_03167_gb300.serve import ALIGN, Arena, percentiles


def test_arena_first_fit_and_coalescing():
    a = Arena(1 << 20)
    x = a.alloc(1000)
    y = a.alloc(5000)
    z = a.alloc(300)
    assert x[0] == 0 and x[1] % ALIGN == 0
    assert y[0] == x[1] and z[0] == x[1] + y[1]
    a.release(y)
    w = a.alloc(4000)            # fits the hole left by y
    assert w[0] == y[0]
    a.release(x)
    a.release(w)
    a.release(z)
    assert a.used == 0
    assert a.free == [(0, 1 << 20)]  # everything coalesced back


def test_arena_never_exceeds_capacity_under_random_load():
    rng = random.Random(5)
    cap = 64 << 20
    a = Arena(cap)
    live = []
    for _ in range(20000):
        if live and rng.random() < 0.45:
            a.release(live.pop(rng.randrange(len(live))))
        else:
            blk = a.alloc(rng.randint(1, 4 << 20))
            if blk is not None:
                live.append(blk)
        assert 0 <= a.used <= cap
        # blocks never overlap
    spans = sorted(live)
    for (o1, s1), (o2, _) in zip(spans, spans[1:]):
        assert o1 + s1 <= o2
    assert a.peak <= cap
    for blk in live:
        a.release(blk)
    assert a.used == 0 and a.free == [(0, cap)]


def test_percentiles():
    p = percentiles(list(range(1, 101)))
    assert abs(p["p50"] - 50.5) < 1e-9 and abs(p["p99"] - 99.01) < 1e-9
    assert percentiles([]) == {"p50": None, "p99": None}
